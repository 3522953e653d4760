// CUDA-core FMA throughput of this GPU (no counterpart in the paper): the
// FP32 / FP64 denominators of the stage kernels' arithmetic roofline.  Every
// thread runs kChains independent fused multiply-add chains (enough
// independent work per warp to cover the FMA latency at full occupancy); the
// host times one launch with CUDA events and counts 2 flops per FMA.
#include <cuda_runtime.h>

#include "dgwedge.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// receives the chains' sum only on an impossible condition (keeps them live)
__device__ double g_fma_sink;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(T a, T b, int iters) {
  T c[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) c[i] = T(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int i = 0; i < kChains; ++i) c[i] = c[i] * a + b;  // contracted to one FMA
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += c[i];
  if (s < T(0)) g_fma_sink = double(s);  // never true: every chain stays positive
}

template <typename T>
int time_fma(cudaStream_t st, int iters, double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return int(e);
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_peak<T>, kThreads, 0);
  if (e != cudaSuccess) return int(e);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) {
    // a = 1 - 2^-20, b = 2^-30: the chains stay finite and the compiler cannot fold them
    const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 1073741824.0);
    k_fma_peak<T><<<grid, kThreads, 0, st>>>(a, b, iters / 8);  // warm-up
    e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) k_fma_peak<T><<<grid, kThreads, 0, st>>>(a, b, iters);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (e != cudaSuccess) return int(e);
  const double flops = 2.0 * kChains * 16.0 * double(iters) * double(grid) * kThreads;
  *tflops = flops / (double(ms) * 1e-3) / 1e12;
  return 0;
}

}  // namespace

extern "C" int dg_fma_peak(int precision, void* stream, double* tflops) {
  if (!tflops || (precision != DG_F32 && precision != DG_F64)) return DG_ERR_ARG;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  // about 10 ms of FP32 work (fewer iterations for the slower FP64 pipe)
  const int rc = precision == DG_F32 ? time_fma<float>(st, 4096, tflops) : time_fma<double>(st, 64, tflops);
  return rc ? DG_ERR_CUDA : DG_OK;
}
