// DG kernels, order N=1, double arithmetic.
#include <cuda_runtime.h>

#include "dg_internal.hpp"

namespace dgw {
namespace f64n1 {
__constant__ AllOps<1, double> c_ops;
}
}  // namespace dgw

#define REAL double
#define REALNS f64n1
#define NORD 1
#include "kernels.cuh"
