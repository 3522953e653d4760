// DG kernels, order N=1, float arithmetic.
#include <cuda_runtime.h>

#include "dg_internal.hpp"

namespace dgw {
namespace f32n1 {
__constant__ AllOps<1, float> c_ops;
}
}  // namespace dgw

#define REAL float
#define REALNS f32n1
#define NORD 1
#include "kernels.cuh"
