// DG kernels, order N=2, float arithmetic.
#include <cuda_runtime.h>

#include "dg_internal.hpp"

namespace dgw {
namespace f32n2 {
__constant__ AllOps<2, float> c_ops;
}
}  // namespace dgw

#define REAL float
#define REALNS f32n2
#define NORD 2
#include "kernels.cuh"
