// Discrete energy of a caller-provided state without any device allocation.
//
// The regular energy path keeps its per-block partial sums in the mesh blob
// the caller allocated at dg_bind.  This translation unit instead holds them
// in a file-scope device array that exists on every GPU that loads the
// library, so the entry point can run where the caller must not allocate
// (inside a framework's allocation-free region, a host callback, or while a
// memory pool is locked).  The state is read in the canonical layout
// [shots][4][total_nodes] (the virtual element of each shot carries its
// shot's canonical offset); geometry and material come from the bound mesh
// blob.  The energy returned is the sum over shots.
#include <cuda_runtime.h>

#include <mutex>

#include "dg_internal.hpp"

namespace dgw {

namespace {

// Per-block partial sums followed by the total: kStaticPartials * 128 elements at most.
__device__ __align__(256) double g_energy_scratch[kStaticPartials + 1];

// Device address of g_energy_scratch per device (0 until set up); written
// once per device under the mutex.
double* g_scratch_ptr[64] = {nullptr};
std::mutex g_scratch_mu;

template <typename real>
__device__ double quad_form(const real* q, int64_t stride, int64_t off, const real* Mmat, int n, int f) {
  double e = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int l = 0; l < n; ++l) s += double(Mmat[i * n + l]) * double(q[f * stride + off + l]);
    e += s * double(q[f * stride + off + i]);
  }
  return e;
}

// One thread per element (wedges first, then tets); E_k = 1/2 (p^T M p / kappa
// + rho sum_c u_c^T M u_c) with the exact (Jacobian-weighted) mass matrices.
template <typename real, int N>
__global__ void __launch_bounds__(128) k_energy_canon(const DevMesh<real> M, const real* __restrict__ q,
                                                      const real* __restrict__ wops, double* scratch) {
  constexpr int Nt = nt_of(N), Nq = N + 1, Npt = npt_of(N);
  const int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t stride = M.total_nodes;
  double E = 0.0;
  if (k < M.Kw) {
    const int Kp = M.Kw_pad;
    const int e = int(k);
    const real* Ma = wops;                 // 3 x Nt x Nt barycentric-weighted masses
    const real* M1 = wops + 3 * Nt * Nt;   // Nq x Nq line mass
    const int v0 = M.w_vid[0 * Kp + e], v1 = M.w_vid[1 * Kp + e], v2 = M.w_vid[2 * Kp + e];
    const double x0 = M.vx[v0], y0 = M.vy[v0];
    const double A = 0.25 * ((double(M.vx[v1]) - x0) * (double(M.vy[v2]) - y0) - (double(M.vx[v2]) - x0) * (double(M.vy[v1]) - y0));
    double Ja[3];
    for (int a = 0; a < 3; ++a)
      Ja[a] = 0.5 * A * (double(M.vz[M.w_vid[(3 + a) * Kp + e]]) - double(M.vz[M.w_vid[a * Kp + e]]));
    const int64_t off = M.w_canon[e];
    for (int f = 0; f < 4; ++f) {
      double ef = 0.0;
      for (int jp = 0; jp < Nq; ++jp)
        for (int jj = 0; jj < Nq; ++jj) {
          double d = 0.0;
          for (int i = 0; i < Nt; ++i) {
            double s = 0.0;
            for (int l = 0; l < Nt; ++l) {
              const double mt = Ja[0] * double(Ma[i * Nt + l]) + Ja[1] * double(Ma[Nt * Nt + i * Nt + l]) +
                                Ja[2] * double(Ma[2 * Nt * Nt + i * Nt + l]);
              s += mt * double(q[f * stride + off + jp * Nt + l]);
            }
            d += double(q[f * stride + off + jj * Nt + i]) * s;
          }
          ef += double(M1[jj * Nq + jp]) * d;
        }
      E += (f == 0 ? 1.0 / double(M.w_mat[0 * Kp + e]) : 1.0 / double(M.w_mat[1 * Kp + e])) * ef;
    }
  } else if (k < int64_t(M.Kw) + M.Kt) {
    const int Kp = M.Kt_pad;
    const int e = int(k - M.Kw);
    double X[4][3];
    for (int v = 0; v < 4; ++v) {
      const int id = M.t_vid[v * Kp + e];
      X[v][0] = M.vx[id];
      X[v][1] = M.vy[id];
      X[v][2] = M.vz[id];
    }
    double G[3][3];
    for (int d = 0; d < 3; ++d)
      for (int m = 0; m < 3; ++m) G[d][m] = 0.5 * (X[m + 1][d] - X[0][d]);
    const double J = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) - G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                     G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
    const int64_t off = M.t_canon[e];
    for (int f = 0; f < 4; ++f) {
      const double w = (f == 0) ? 1.0 / double(M.t_mat[0 * Kp + e]) : 1.0 / double(M.t_mat[1 * Kp + e]);
      E += w * J * quad_form(q, stride, off, M.tet_mass, Npt, f);
    }
  }
  __shared__ double red[128];
  red[threadIdx.x] = E;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) scratch[blockIdx.x] = 0.5 * red[0];
}

__global__ void k_energy_canon_final(double* scratch, int n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += scratch[i];
    scratch[kStaticPartials] = s;
  }
}

template <typename real, int N>
int launch(const DevMesh<real>& m, const real* q, const real* wops, double* scratch, int nblocks, cudaStream_t s) {
  k_energy_canon<real, N><<<nblocks, 128, 0, s>>>(m, q, wops, scratch);
  k_energy_canon_final<<<1, 32, 0, s>>>(scratch, nblocks);
  return int(cudaGetLastError());
}

}  // namespace

// One-time, per-device set-up: the device address of the scratch array (the
// array's name in host code is only a host-side stand-in).  The address is
// looked up with `device` current -- the call refuses to run with another
// device current, so a wrong device's address can never be cached -- and kept
// per device; concurrent first calls from several host threads are
// serialised.  The first dg_energy_static call on a device performs it.
int energy_static_scratch(int device, double** out) {
  if (device < 0 || device >= 64) return int(cudaErrorInvalidDevice);
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return int(e);
  if (cur != device) return int(cudaErrorInvalidDevice);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess) return int(e);
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return 0;
}

template <typename real>
int launch_energy_static(int N, const DevMesh<real>& m, const real* q, const real* wops, double* scratch, int nblocks,
                         void* stream) {
  const cudaStream_t s = cudaStream_t(stream);
  switch (N) {
    case 1: return launch<real, 1>(m, q, wops, scratch, nblocks, s);
    case 2: return launch<real, 2>(m, q, wops, scratch, nblocks, s);
    case 3: return launch<real, 3>(m, q, wops, scratch, nblocks, s);
    case 4: return launch<real, 4>(m, q, wops, scratch, nblocks, s);
    case 5: return launch<real, 5>(m, q, wops, scratch, nblocks, s);
  }
  return int(cudaErrorInvalidValue);
}
template int launch_energy_static<float>(int, const DevMesh<float>&, const float*, const float*, double*, int, void*);
template int launch_energy_static<double>(int, const DevMesh<double>&, const double*, const double*, double*, int,
                                          void*);

}  // namespace dgw
