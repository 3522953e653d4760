// DG kernels, order N=3, double arithmetic.
#include <cuda_runtime.h>

#include "dg_internal.hpp"

namespace dgw {
namespace f64n3 {
__constant__ AllOps<3, double> c_ops;
}
}  // namespace dgw

#define REAL double
#define REALNS f64n3
#define NORD 3
#include "kernels.cuh"
