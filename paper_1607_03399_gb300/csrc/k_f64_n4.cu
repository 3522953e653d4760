// DG kernels, order N=4, double arithmetic.
#include <cuda_runtime.h>

#include "dg_internal.hpp"

namespace dgw {
namespace f64n4 {
__constant__ AllOps<4, double> c_ops;
}
}  // namespace dgw

#define REAL double
#define REALNS f64n4
#define NORD 4
#include "kernels.cuh"
