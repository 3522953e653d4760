// DG kernels, order N=3, float arithmetic.
#include <cuda_runtime.h>

#include "dg_internal.hpp"

namespace dgw {
namespace f32n3 {
__constant__ AllOps<3, float> c_ops;
}
}  // namespace dgw

#define REAL float
#define REALNS f32n3
#define NORD 3
#include "kernels.cuh"
