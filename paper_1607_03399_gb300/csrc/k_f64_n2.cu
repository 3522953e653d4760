// DG kernels, order N=2, double arithmetic.
#include <cuda_runtime.h>

#include "dg_internal.hpp"

namespace dgw {
namespace f64n2 {
__constant__ AllOps<2, double> c_ops;
}
}  // namespace dgw

#define REAL double
#define REALNS f64n2
#define NORD 2
#include "kernels.cuh"
