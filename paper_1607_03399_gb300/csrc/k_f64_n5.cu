// DG kernels, order N=5, double arithmetic.
#include <cuda_runtime.h>

#include "dg_internal.hpp"

namespace dgw {
namespace f64n5 {
__constant__ AllOps<5, double> c_ops;
}
}  // namespace dgw

#define REAL double
#define REALNS f64n5
#define NORD 5
#include "kernels.cuh"
