// DG kernels, order N=4, float arithmetic.
#include <cuda_runtime.h>

#include "dg_internal.hpp"

namespace dgw {
namespace f32n4 {
__constant__ AllOps<4, float> c_ops;
}
}  // namespace dgw

#define REAL float
#define REALNS f32n4
#define NORD 4
#include "kernels.cuh"
