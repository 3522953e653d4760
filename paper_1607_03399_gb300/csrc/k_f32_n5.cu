// DG kernels, order N=5, float arithmetic.
#include <cuda_runtime.h>

#include "dg_internal.hpp"

namespace dgw {
namespace f32n5 {
__constant__ AllOps<5, float> c_ops;
}
}  // namespace dgw

#define REAL float
#define REALNS f32n5
#define NORD 5
#include "kernels.cuh"
