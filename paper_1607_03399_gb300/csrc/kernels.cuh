// CUDA kernels of the DG stage (included once per precision; the including
// translation unit defines REAL and the constant-memory table c_ops).
//
// Wedge stage (Sections 3.2, 4.2; one launch per Runge-Kutta stage):
//   CTA = 32 consecutive wedges x (N+1) warps; warp j owns GLL slice j of all
//   32 elements, lane = element.  Per element and slice:
//     geometry from the 6 vertices (Lemma 3.1): r_x, r_y, s_x, s_y, t_zJ = A
//       constant, t_xJ, t_yJ at t_j, J_a = A h_a / 2 at the three columns;
//     W_j = M^tri [ T_j + J_fb ell0_j F_bot + J_ft ellN_j F_top ]
//           + sum_quad M~_e F_e,j                       (lift, weak form)
//       T_j = - sum_c t_cJ(t_j) (D_t u_c)_j  (p),  - t_cJ(t_j) (D_t p)_j  (u_c)
//     X_j = (M^{tri,k})^{-1} W_j, M^{tri,k} = sum_a J_a M_a, by a per-element
//       Cholesky factor computed on the fly (exact inverse of the
//       Jacobian-weighted wedge mass, Section 4.2);
//     rhs = kappa (-(D_r (r.u) + D_s (s.u))_j + X_p),
//     rhs_u_c = (1/rho) (-(r_c D_r p + s_c D_s p)_j + X_u_c);
//     fused LSRK update res <- a res + dt rhs, q_out <- q_in + b res.
// Tet stage: affine tets, one thread per element (Section 3.2: physical
//   operators are scaled reference operators).
#pragma once
#include <cuda_runtime.h>
#include <type_traits>

#include "dg_internal.hpp"

namespace dgw {
namespace REALNS {

using real = REAL;

template <int N>
__device__ __forceinline__ const AllOps<N, real>& OPS() {
  static_assert(N == NORD, "one order per translation unit");
  return c_ops;
}

__device__ __forceinline__ float rsqrt_r(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_r(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }

// triangle node (a, b) -> index; edge node m of triangle edge ed (from its
// first to its second vertex)
__host__ __device__ constexpr int tri_idx(int N, int a, int b) { return b * (N + 1) - (b * (b - 1)) / 2 + a; }
__host__ __device__ constexpr int edge_node(int N, int ed, int m) {
  return ed == 0 ? tri_idx(N, m, 0) : (ed == 1 ? tri_idx(N, N - m, m) : tri_idx(N, 0, N - m));
}
// k-th node of tet face f in element node order
__host__ __device__ constexpr int tet_face_node(int N, int f, int k) {
  int n = 0, cnt = 0;
  for (int c = 0; c <= N; ++c)
    for (int b = 0; b <= N - c; ++b)
      for (int a = 0; a <= N - b - c; ++a) {
        const bool on = (f == 0) ? (c == 0) : (f == 1) ? (b == 0) : (f == 2) ? (a + b + c == N) : (a == 0);
        if (on) {
          if (cnt == k) return n;
          ++cnt;
        }
        ++n;
      }
  return -1;
}

// Packed state layout: node-major, the four fields innermost, so one thread
// moves a node's (p, u_x, u_y, u_z) with one 16-byte (FP32) access and a warp
// moves 512 contiguous bytes:
//   wedge region [nblk_w][Np][32 lanes][4 fields], tet region likewise.
template <int N>
__device__ __forceinline__ int64_t widx(int blk_e, int node, int lane) {
  constexpr int Np = npw_of(N);
  return ((int64_t(blk_e) * Np + node) * kB + lane) * 4;
}
template <int N>
__device__ __forceinline__ int64_t tidx(int64_t off, int blk_e, int node, int lane) {
  constexpr int Np = npt_of(N);
  return off + ((int64_t(blk_e) * Np + node) * kB + lane) * 4;
}

struct Q4 {
  real p, u, v, w;
};
__device__ __forceinline__ Q4 q4_from(const float4 t) { return Q4{real(t.x), real(t.y), real(t.z), real(t.w)}; }
// shared-memory slab [Np][32][4]
__device__ __forceinline__ Q4 lds4(const real* slab, int node, int lane) {
  const real* a = slab + ((node * kB + lane) << 2);
  if constexpr (sizeof(real) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(a);
    return Q4{real(t.x), real(t.y), real(t.z), real(t.w)};
  } else {
    const double2 t0 = reinterpret_cast<const double2*>(a)[0], t1 = reinterpret_cast<const double2*>(a)[1];
    return Q4{real(t0.x), real(t0.y), real(t1.x), real(t1.y)};
  }
}
// global, read-only for the kernel's lifetime (the stage input)
__device__ __forceinline__ Q4 ldg4(const real* __restrict__ q, int64_t idx) {
  if constexpr (sizeof(real) == 4) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(q + idx));
    return Q4{real(t.x), real(t.y), real(t.z), real(t.w)};
  } else {
    const double2 t0 = __ldg(reinterpret_cast<const double2*>(q + idx));
    const double2 t1 = __ldg(reinterpret_cast<const double2*>(q + idx) + 1);
    return Q4{real(t0.x), real(t0.y), real(t1.x), real(t1.y)};
  }
}
// global, coherent (the residual, rewritten by the same thread)
__device__ __forceinline__ Q4 ld4(const real* q, int64_t idx) {
  if constexpr (sizeof(real) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(q + idx);
    return Q4{real(t.x), real(t.y), real(t.z), real(t.w)};
  } else {
    const double2 t0 = reinterpret_cast<const double2*>(q + idx)[0], t1 = reinterpret_cast<const double2*>(q + idx)[1];
    return Q4{real(t0.x), real(t0.y), real(t1.x), real(t1.y)};
  }
}
// generic address: the block's slab in shared memory or the stage input in global memory
__device__ __forceinline__ Q4 ldx4(const real* a) {
  if constexpr (sizeof(real) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(a);
    return Q4{real(t.x), real(t.y), real(t.z), real(t.w)};
  } else {
    const double2 t0 = reinterpret_cast<const double2*>(a)[0], t1 = reinterpret_cast<const double2*>(a)[1];
    return Q4{real(t0.x), real(t0.y), real(t1.x), real(t1.y)};
  }
}
// shared-memory operator records: (a, b, c, d) in natural order -> Q4{a, b, c, d}
__device__ __forceinline__ Q4 ldop4(const real* a) {
  if constexpr (sizeof(real) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(a);
    return Q4{real(t.x), real(t.y), real(t.z), real(t.w)};
  } else {
    const double2 t0 = reinterpret_cast<const double2*>(a)[0], t1 = reinterpret_cast<const double2*>(a)[1];
    return Q4{real(t0.x), real(t0.y), real(t1.x), real(t1.y)};
  }
}
__device__ __forceinline__ void ldop2(const real* a, real& x, real& y) {
  if constexpr (sizeof(real) == 4) {
    const float2 t = *reinterpret_cast<const float2*>(a);
    x = real(t.x);
    y = real(t.y);
  } else {
    const double2 t = *reinterpret_cast<const double2*>(a);
    x = real(t.x);
    y = real(t.y);
  }
}
__device__ __forceinline__ void st4(real* q, int64_t idx, const Q4& v) {
  if constexpr (sizeof(real) == 4) {
    *reinterpret_cast<float4*>(q + idx) = make_float4(float(v.p), float(v.u), float(v.v), float(v.w));
  } else {
    reinterpret_cast<double2*>(q + idx)[0] = make_double2(double(v.p), double(v.u));
    reinterpret_cast<double2*>(q + idx)[1] = make_double2(double(v.v), double(v.w));
  }
}

// Packed pairs.  In FP32 one packed FMA instruction (sm_100 family) performs
// two multiply-adds, each rounded as fmaf: half the issue slots of the scalar
// form, same results.  In FP64 a pair is two scalar FMAs.
using real2 = typename std::conditional<sizeof(real) == 4, float2, double2>::type;
__device__ __forceinline__ float2 fma2(const float2 a, const float2 b, const float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 fma2(const double2 a, const double2 b, const double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 add2(const float2 a, const float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 add2(const double2 a, const double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 mul2(const float2 a, const float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 mul2(const double2 a, const double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ real2 dup2(const real v) {
  real2 r;
  r.x = v;
  r.y = v;
  return r;
}
__device__ __forceinline__ real2 mk2(const real a, const real b) {
  real2 r;
  r.x = a;
  r.y = b;
  return r;
}
// entry (h, l) of an output-pair table (constant memory; an 8-byte operand)
__device__ __forceinline__ real2 cpair(const real* XP, int cols, int h, int l) {
  return *reinterpret_cast<const real2*>(XP + (h * cols + l) * 2);
}
// acc = X x for an NR x NC operator given by output pairs XP (acc[h] holds
// rows 2h, 2h + 1): every output accumulates its products over l in order
template <int NR, int NC>
__device__ __forceinline__ void apply_pairs(const real* XP, const real (&x)[NC], real2 (&acc)[(NR + 1) / 2]) {
  constexpr int NH = (NR + 1) / 2;
#pragma unroll
  for (int h = 0; h < NH; ++h) acc[h] = dup2(real(0));
#pragma unroll
  for (int l = 0; l < NC; ++l) {
    const real2 xx = dup2(x[l]);
#pragma unroll
    for (int h = 0; h < NH; ++h) acc[h] = fma2(cpair(XP, NC, h, l), xx, acc[h]);
  }
}
// row i of a pair-accumulated result
__device__ __forceinline__ real pair_row(const real2* acc, int i) { return (i & 1) ? acc[i >> 1].y : acc[i >> 1].x; }

// a * b + c rounded once (an explicit FMA: the same rounding wherever the
// compiler places the expression, so kernel variants that differ only in when
// they load the operands give the same bits)
__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmar(double a, double b, double c) { return fma(a, b, c); }
// Penalty fluxes of eq. (1): F_p = 1/2 (tau_p [p] - [u_n]), F_u = 1/2 (tau_u [u_n] - [p]).
__device__ __forceinline__ void penalty_flux(real dp, real dun, real tau_p, real tau_u, real& Fp, real& Fu) {
  Fp = real(0.5) * fmar(tau_p, dp, -dun);
  Fu = real(0.5) * fmar(tau_u, dun, -dp);
}
// Boundary ghosts: Dirichlet p+ = -p-, u+ = u-  -> [p] = -2p, [u_n] = 0;
// rigid p+ = p-, u+ = u- - 2 u_n n             -> [p] = 0, [u_n] = -2 u_n.
__device__ __forceinline__ void boundary_jumps(int bc, real pM, real unM, real& dp, real& dun) {
  const bool dir = bc == 0;
  dp = dir ? real(-2) * pM : real(0);
  dun = dir ? real(0) : real(-2) * unM;
}

__device__ __forceinline__ void taus(int flux, real zM, real zP, real& tau_p, real& tau_u) {
  const real zavg = real(0.5) * (zM + zP);
  const real izavg = real(1) / zavg;
  const bool up = flux == 0;
  tau_p = up ? izavg : real(0);
  tau_u = up ? zavg : real(0);
}

// ---------------------------------------------------------------------------
// shared reference operators on the tensor cores (FP32 fields, warp-level
// mma.sync): Out = Op * In with Op an Nt x Nt triangle operator zero-padded
// to 16 x 16 (the A operand, in registers) and In an Nt-row tile in shared
// memory whose columns are (element, field) pairs (the B operand).  TF32 is
// m16n8k8 (two k-steps cover Nt <= 16), BF16 m16n8k16 (one k-step); both
// accumulate in FP32.  3xTF32 splits each operand x = hi + lo into two TF32
// numbers and adds lo*hi + hi*lo + hi*hi (dropping lo*lo), which recovers
// about FP32 accuracy.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// (lo, hi) -> bf16x2 with lo in the low half (the lower k index of an operand pair)
__device__ __forceinline__ uint32_t bf16x2_of(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A operand registers of one operator: [k-step][4] (hi and, for 3xTF32, lo parts)
template <int OP>
struct AFrag {
  uint32_t h[2][4];
  uint32_t l[OP == kOpTF32x3 ? 2 : 1][4];
};
// Fragment of the row-major Nt x Nt operator Op (rows = outputs), zero-padded.
// m16n8k8 TF32: a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4) of
// the 16 x 8 slice of k-step ks; m16n8k16 BF16: pairs of columns (2t, 2t + 1)
// and (2t + 8, 2t + 9) of rows g and g + 8 (g = lane / 4, t = lane % 4).
template <int NT, int OP>
__device__ __forceinline__ void afrag_load(const float* Op, int lane, AFrag<OP>& A) {
  const int g = lane >> 2, t = lane & 3;
  auto at = [&](int r, int c) -> float { return (r < NT && c < NT) ? Op[r * NT + c] : 0.f; };
  if constexpr (OP == kOpBF16) {
    A.h[0][0] = bf16x2_of(at(g, 2 * t), at(g, 2 * t + 1));
    A.h[0][1] = bf16x2_of(at(g + 8, 2 * t), at(g + 8, 2 * t + 1));
    A.h[0][2] = bf16x2_of(at(g, 2 * t + 8), at(g, 2 * t + 9));
    A.h[0][3] = bf16x2_of(at(g + 8, 2 * t + 8), at(g + 8, 2 * t + 9));
  } else {
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      const float v[4] = {at(g, t + 8 * ks), at(g + 8, t + 8 * ks), at(g, t + 4 + 8 * ks), at(g + 8, t + 4 + 8 * ks)};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        A.h[ks][r] = tf32_of(v[r]);
        if constexpr (OP == kOpTF32x3) A.l[ks][r] = tf32_of(v[r] - __uint_as_float(A.h[ks][r]));
      }
    }
  }
}
// B operand of one n-tile: column `col` of the Nt-row operand tile B (layout
// tile_at); rows >= Nt are zero (never read).  TF32: [k-step] (k = t, t + 4)
// per step; BF16: (2t, 2t + 1) and (2t + 8, 2t + 9).
template <int OP>
struct BFrag {
  uint32_t h[2][2];
  uint32_t l[OP == kOpTF32x3 ? 2 : 1][2];
};
template <int NT, int OP>
__device__ __forceinline__ void bfrag_load(const float* B, int col, int lane, BFrag<OP>& F) {
  const int t = lane & 3;
  auto bv = [&](int k) -> float { return k < NT ? B[tile_at(k, col)] : 0.f; };
  if constexpr (OP == kOpBF16) {
    F.h[0][0] = bf16x2_of(bv(2 * t), bv(2 * t + 1));
    F.h[0][1] = bf16x2_of(bv(2 * t + 8), bv(2 * t + 9));
  } else {
#pragma unroll
    for (int ks = 0; ks < (NT + 7) / 8; ++ks) {
      const float x0 = bv(t + 8 * ks), x1 = bv(t + 4 + 8 * ks);
      F.h[ks][0] = tf32_of(x0);
      F.h[ks][1] = tf32_of(x1);
      if constexpr (OP == kOpTF32x3) {
        F.l[ks][0] = tf32_of(x0 - __uint_as_float(F.h[ks][0]));
        F.l[ks][1] = tf32_of(x1 - __uint_as_float(F.h[ks][1]));
      }
    }
  }
}
// d += Op * B for one 16 x 8 output tile
template <int NT, int OP>
__device__ __forceinline__ void op_mma(const AFrag<OP>& A, const BFrag<OP>& F, float (&d)[4]) {
  if constexpr (OP == kOpBF16) {
    mma_bf16(d, A.h[0], F.h[0][0], F.h[0][1]);
  } else {
#pragma unroll
    for (int ks = 0; ks < (NT + 7) / 8; ++ks) {
      if constexpr (OP == kOpTF32x3) {
        mma_tf32(d, A.l[ks], F.h[ks][0], F.h[ks][1]);
        mma_tf32(d, A.h[ks], F.l[ks][0], F.l[ks][1]);
      }
      mma_tf32(d, A.h[ks], F.h[ks][0], F.h[ks][1]);
    }
  }
}

// Ricker wavelet (1 - 2 a) exp(-a), a = (pi f0 (t - t0))^2 (c13 reading).
__device__ __forceinline__ double ricker(double f0, double tau) {
  const double a = (3.14159265358979323846 * f0 * tau) * (3.14159265358979323846 * f0 * tau);
  return (1.0 - 2.0 * a) * exp(-a);
}
// True when a point source lies in element (type, elem): the entries, sorted by
// element, of its 32-element block are scanned.
__device__ __forceinline__ bool has_source(const DevMesh<real>& M, int type, int elem) {
  const int* rng = (type == 6 ? M.w_srng : M.t_srng) + 2 * (elem >> 5);
  const int b = rng[0], e = rng[1];
  for (int s = b; s < e; ++s)
    if (M.src[s].elem == elem) return true;
  return false;
}
// Point-source forcing of element (type, elem) at time t added to the pressure
// accumulators acc[c] of element nodes n0 + c (c < C, n0 + c < np), before the
// kappa scaling: acc += w_s(t) g_s with g_s = (M^k)^{-1} l(x_s) and w_s the
// source's Ricker amplitude.  The time function is evaluated once per source.
template <int C>
__device__ __forceinline__ void add_sources(const DevMesh<real>& M, int type, int elem, int n0, int np, double t,
                                            real (&acc)[C]) {
  const int* rng = (type == 6 ? M.w_srng : M.t_srng) + 2 * (elem >> 5);
  const int sb = rng[0], se = rng[1];
#pragma unroll 1
  for (int s = sb; s < se; ++s) {
    const SourceDev& sd = M.src[s];
    if (sd.elem != elem) continue;
    const real w = real(sd.amp * ricker(sd.f0, t - sd.t0));
    const real* __restrict__ g = M.src_g + sd.goff + n0;
#pragma unroll
    for (int c = 0; c < C; ++c)
      if (n0 + c < np) acc[c] += w * g[c];
  }
}
// the same on field-pair accumulators whose x component is the pressure
template <int C>
__device__ __forceinline__ void add_sources(const DevMesh<real>& M, int type, int elem, int n0, int np, double t,
                                            real2 (&acc)[C]) {
  const int* rng = (type == 6 ? M.w_srng : M.t_srng) + 2 * (elem >> 5);
  const int sb = rng[0], se = rng[1];
#pragma unroll 1
  for (int s = sb; s < se; ++s) {
    const SourceDev& sd = M.src[s];
    if (sd.elem != elem) continue;
    const real w = real(sd.amp * ricker(sd.f0, t - sd.t0));
    const real* __restrict__ g = M.src_g + sd.goff + n0;
#pragma unroll
    for (int c = 0; c < C; ++c)
      if (n0 + c < np) acc[c].x += w * g[c];
  }
}

__global__ void k_clock(double* clock, double dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *clock += dt;
}
// sets the device clock (state loads: no host staging, so no synchronisation)
__global__ void k_set_clock(double* clock, double t) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *clock = t;
}

// ---------------------------------------------------------------------------
// wedge stage
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// bulk asynchronous copies (TMA engine) with mbarrier completion; every wait
// is bounded and reports a timeout through the device error word
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// One poll of the phase; the thread may be suspended for up to the hint
// (1 us) while the phase is incomplete, so waiting threads do not spin.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase), "n"(1000)
      : "memory");
  return ok != 0;
}
// About a second of polling at most (each poll suspends for at most ~1 us).
constexpr long long kWaitLimit = 1ll << 20;
template <long long Limit = kWaitLimit>
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  for (long long it = 0; it < Limit; ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

// Failure-path check: one warp arms an mbarrier for bytes that no copy will
// ever deliver (no copy is issued), so the stages' bounded wait runs out --
// here after 64 polls instead of the stages' ~1 s budget -- and the kernel
// reports DG_ERR_TIMEOUT through the device error word, exactly as a stage
// whose copy never landed does, then returns.  Nothing is in flight when it
// exits; the GPU and the context stay usable.
__global__ void k_wait_expire(int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_expect_tx(&bar, 16u);
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded<64>(&bar, 0));
  if (!ok && threadIdx.x == 0) atomicOr(err, kErrTimeout);
}

// per-element geometric factors kept in shared memory ([item][32])
// (the column Jacobians J0..J2 come last: the stage does not use them and
// keeps only the first G_STAGE items)
enum WGeo : int {
  G_RX, G_RY, G_SX, G_SY, G_A, G_NB0, G_NB1, G_NB2, G_NT0, G_NT1, G_NT2, G_JFB, G_JFT,
  G_QNX0, G_QNX1, G_QNX2, G_QNY0, G_QNY1, G_QNY2, G_QCA0, G_QCA1, G_QCA2, G_QCB0, G_QCB1, G_QCB2,
  G_TX0, G_TX1, G_TY0, G_TY1, G_STAGE, G_J0 = G_STAGE, G_J1, G_J2, G_COUNT
};

// Residual slab staged in shared memory by the bulk copy (FP32 up to N = 4,
// FP64 up to N = 3), so that the update reads it there instead of one
// dependent global load per node at the end of the kernel.  At N = 4 the
// stage runs two CTAs per SM (registers), and 103 KB of shared memory per CTA
// still fits two: with the packed-pair arithmetic the staged slab measured
// 1075 -> 820 us per stage on 524,288 wedges (before it, with the scalar
// arithmetic, it had measured slower).  With tensor-core applies the operand
// tiles (Nq x Nt x 128 reals, the size of the residual slab) share the
// residual slab's space: the residual is copied in once the weak-form
// accumulation has released them.
template <int N, int OP = kOpFFMA>
__host__ __device__ constexpr bool stage_res() {
  return sizeof(real) == 4 ? N <= 4 : N <= 3;
}

template <int N, int OP = kOpFFMA>
struct WedgeSmem {
  static constexpr int Nt = nt_of(N), Nq = N + 1, Np = Nt * Nq;
  static constexpr int q = 0;                                            // [4][Np][32]
  static constexpr int r = q + 4 * Np * kB;                              // [4][Np][32] (if staged)
  static constexpr int L = r + (stage_res<N, OP>() ? 4 * Np * kB : 0);   // [NL4][32][4]
  static constexpr int F = L + nl4_of(N) * 4 * kB;                        // [4][Nt][32]
  static constexpr int G = F + 4 * Nt * kB;                              // [G_STAGE][32]
  // per-warp operand tiles [Nt][kTP] (tensor cores): the residual slab's space where it is staged
  static constexpr int T = stage_res<N, OP>() ? r : G + G_STAGE * kB;
  static constexpr int reals = G + G_STAGE * kB + ((OP == kOpFFMA || stage_res<N, OP>()) ? 0 : Nq * Nt * kTP);
};

template <int N, int OP = kOpFFMA>
__host__ __device__ constexpr int wedge_smem_reals() {
  return WedgeSmem<N, OP>::reals;
}
// Element blocks per CTA.  The warps that work on slice j of the CTA's blocks
// share an SM sub-partition and run the same straight-line code side by side,
// so they share its instruction cache lines.  With the mass factor computed in
// the stage (a long serial factorisation on one warp per block) two blocks per
// CTA measured faster at N = 3 FP32; with the stored factor, one.
template <int N>
__host__ __device__ constexpr int wedge_bpc_onthefly() {
  return (sizeof(real) == 4 && N == 3) ? 2 : 1;
}
// bytes: per block two mbarriers and a status word (32 bytes), then per block
// the reals (each block's slabs start 16-byte aligned)
template <int N, int BPC, int OP = kOpFFMA>
__host__ __device__ constexpr int wedge_smem_bytes() {
  return BPC * (32 + wedge_smem_reals<N, OP>() * int(sizeof(real)));
}
// resident CTAs per SM the stage is compiled for
template <int N, int BPC, int OP>
__host__ __device__ constexpr int wedge_min_ctas() {
  return sizeof(REAL) == 4 ? (N >= 4 ? 2 : 4 / BPC) : 1;
}

// Lemma 3.1 for one wedge: everything the stage needs, from the six vertices
// (bi-unit reference, x = sum_a lambda_a(r,s) [(1-t)/2 X_a + (1+t)/2 X_{a+3}]),
// X = [x_a][y_a][zb_a][zt_a] (a = 0..2, bottom x and y; bottom and top z).
__device__ __forceinline__ void wedge_geometry_vals(const real (&X)[12], real (&G)[G_COUNT]) {
  const real x0 = X[0], x1 = X[1], x2 = X[2], y0 = X[3], y1 = X[4], y2 = X[5];
  const real zb0 = X[6], zb1 = X[7], zb2 = X[8], zt0 = X[9], zt1 = X[10], zt2 = X[11];
  const real xr = real(0.5) * (x1 - x0), xs = real(0.5) * (x2 - x0);
  const real yr = real(0.5) * (y1 - y0), ys = real(0.5) * (y2 - y0);
  const real A = xr * ys - xs * yr;  // t_z J (constant)
  const real iA = real(1) / A;
  G[G_RX] = ys * iA;
  G[G_RY] = -xs * iA;
  G[G_SX] = -yr * iA;
  G[G_SY] = xr * iA;
  G[G_A] = A;
  const real h0 = zt0 - zb0, h1 = zt1 - zb1, h2 = zt2 - zb2;
  G[G_J0] = real(0.5) * A * h0;  // J at the three columns (J linear in r, s)
  G[G_J1] = real(0.5) * A * h1;
  G[G_J2] = real(0.5) * A * h2;
  // z_r, z_s are linear in t: z_r(t) = zr0 + t zr1 (likewise z_s), so
  // t_x J = y_r z_s - z_r y_s and t_y J = z_r x_s - x_r z_s are linear in t
  const real zr0 = real(0.25) * ((zb1 - zb0) + (zt1 - zt0)), zr1 = real(0.25) * ((zt1 - zt0) - (zb1 - zb0));
  const real zs0 = real(0.25) * ((zb2 - zb0) + (zt2 - zt0)), zs1 = real(0.25) * ((zt2 - zt0) - (zb2 - zb0));
  G[G_TX0] = yr * zs0 - zr0 * ys;
  G[G_TX1] = yr * zs1 - zr1 * ys;
  G[G_TY0] = zr0 * xs - xr * zs0;
  G[G_TY1] = zr1 * xs - xr * zs1;
  {
    // triangle faces: n = c / |c| with c the edge cross product, J_f = |c| / 4
    const real ax = x1 - x0, ay = y1 - y0, bx = x2 - x0, by = y2 - y0;
    real az = zb1 - zb0, bz = zb2 - zb0;
    real cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
    real cc = cx * cx + cy * cy + cz * cz, ic = rsqrt_r(cc);
    G[G_JFB] = real(0.25) * cc * ic;
    G[G_NB0] = -cx * ic;
    G[G_NB1] = -cy * ic;
    G[G_NB2] = -cz * ic;
    az = zt1 - zt0;
    bz = zt2 - zt0;
    cx = ay * bz - az * by;
    cy = az * bx - ax * bz;
    cz = ax * by - ay * bx;
    cc = cx * cx + cy * cy + cz * cz;
    ic = rsqrt_r(cc);
    G[G_JFT] = real(0.25) * cc * ic;
    G[G_NT0] = cx * ic;
    G[G_NT1] = cy * ic;
    G[G_NT2] = cz * ic;
  }
  const real xx[3] = {x0, x1, x2}, yy[3] = {y0, y1, y2}, hh[3] = {h0, h1, h2};
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) {
    const int ia = ed, ib = (ed + 1) % 3;
    const real dx = xx[ib] - xx[ia], dy = yy[ib] - yy[ia];
    const real ll = dx * dx + dy * dy, il = rsqrt_r(ll);
    const real Le = ll * il;
    G[G_QNX0 + ed] = dy * il;  // horizontal outward normal of the quad face
    G[G_QNY0 + ed] = -dx * il;
    G[G_QCA0 + ed] = real(0.25) * Le * hh[ia];  // M~_e = ca Mea + cb Meb
    G[G_QCB0 + ed] = real(0.25) * Le * hh[ib];
  }
}

// The stage's geometry warp: coordinates arrive in the first 12 items of the
// shared table (one column per lane) and are replaced by the first NG factors.
template <int NG = G_COUNT>
__device__ __forceinline__ void wedge_geometry(real* sG, int lane) {
  real X[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) X[i] = sG[i * kB + lane];
  __syncwarp();
  real G[G_COUNT];
  wedge_geometry_vals(X, G);
#pragma unroll
  for (int i = 0; i < NG; ++i) sG[i * kB + lane] = G[i];
}

// TF: the neighbour nodes of the triangle-face fluxes are requested before the
// quadrilateral faces (one block per CTA: meshes where some of them are tets
// or lie in another block, StageArgs::tri_far; two blocks per CTA: always);
// otherwise each is read where its flux is formed
template <int N, int BPC, int OP = kOpFFMA, bool TF = false>
__global__ void __launch_bounds__(32 * (N + 1) * BPC, wedge_min_ctas<N, BPC, OP>())
    k_wedge_stage(const StageArgs<real> A, bool rk) {
  constexpr int Nt = nt_of(N), Nq = N + 1, Np = Nt * Nq;
  static_assert(OP == kOpFFMA || (sizeof(real) == 4 && BPC == 1 && Nt <= 16), "tensor-core applies: FP32, Nt <= 16");
  using SM = WedgeSmem<N, OP>;
  const AllOps<N, real>& O = OPS<N>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // block sb of this CTA: warps sb (N+1) .. sb (N+1) + N, one per slice
  const int sb = threadIdx.x / (32 * Nq);
  const int j = (threadIdx.x >> 5) - sb * Nq;
  const bool leader = int(threadIdx.x) == sb * 32 * Nq;
  // [0] state slab (and stored factor), [1] residual slab, [2] vertex coordinates
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 32 * sb);
  int* status = reinterpret_cast<int*>(smem_raw + 32 * sb + 24);
  real* base = reinterpret_cast<real*>(smem_raw + 32 * BPC) + sb * SM::reals;
  real* sq = base + SM::q;
  real* sr = base + SM::r;
  real* sL = base + SM::L;
  real* sF = base + SM::F;
  real* sG = base + SM::G;
  real* sT = base + SM::T + j * Nt * kTP;  // this warp's operand tile (tensor cores)
  const DevMesh<real>& M = A.m;
  const real* __restrict__ qin = A.q_in;
  real* __restrict__ qout = A.q_out;
  real* __restrict__ resg = A.res;
  const int lane = threadIdx.x & 31;
  const int blk = blockIdx.x * BPC + sb;
  const bool live = blk < M.nblk_w;  // false only for padding blocks of the last CTA
  const int e = blk * kB + lane;
  const int Kp = M.Kw_pad;
  constexpr uint32_t slab_bytes = uint32_t(4 * Np * kB * sizeof(real));
  const bool res_async = rk && stage_res<N, OP>();
  // the residual copy is issued with the state's (FP32 FMA applies) or after
  // the weak-form accumulation, once the operand tiles in its space are free
  const bool res_early = res_async && OP == kOpFFMA;
#define GEO(item) sG[(item) * kB + lane]
#define LQ(q) sL[(((q) >> 2) * kB + lane) * 4 + ((q) & 3)]

  if (!live) return;  // padding block of the last CTA
  // the warps of one block synchronise among themselves (named barrier 1 + sb)
  // (immediate barrier ids, so that only BPC + 1 hardware barriers are reserved)
  auto block_sync = [&]() {
    static_assert(BPC <= 4, "at most four blocks per CTA");
    if (sb == 0) asm volatile("bar.sync 1, %0;" ::"n"(32 * Nq) : "memory");
    else if (BPC > 1 && sb == 1) asm volatile("bar.sync 2, %0;" ::"n"(32 * Nq) : "memory");
    else if (BPC > 2 && sb == 2) asm volatile("bar.sync 3, %0;" ::"n"(32 * Nq) : "memory");
    else if (BPC > 3) asm volatile("bar.sync 4, %0;" ::"n"(32 * Nq) : "memory");
  };
  // 0. bulk copies of the block's state (and residual) slabs; geometry meanwhile
  constexpr int NL4 = nl4_of(N);
  constexpr uint32_t fac_bytes = uint32_t(NL4 * 4 * kB * sizeof(real));
  const bool stored = M.w_fac != nullptr;
  constexpr uint32_t xyz_bytes = uint32_t(12 * kB * sizeof(real));
  if (leader) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    mbar_init(&bar[3], 1);
    fence_mbar_init();
    // the block's vertex coordinates first (the geometry warp waits on them alone)
    mbar_expect_tx(&bar[2], xyz_bytes);
    bulk_g2s(sG, M.w_xyz + int64_t(blk) * 12 * kB, xyz_bytes, &bar[2]);
    mbar_expect_tx(&bar[0], slab_bytes + (stored ? fac_bytes : 0u));
    bulk_g2s(sq, qin + int64_t(blk) * 4 * Np * kB, slab_bytes, &bar[0]);
    // stored mass factor: straight into the factor table with the state slab
    if (stored) bulk_g2s(sL, M.w_fac + int64_t(blk) * NL4 * 4 * kB, fac_bytes, &bar[0]);
    if (res_early) {
      mbar_expect_tx(&bar[1], slab_bytes);
      bulk_g2s(sr, resg + int64_t(blk) * 4 * Np * kB, slab_bytes, &bar[1]);
    }
  }
  // face neighbours, their impedances and the source flag, loaded while the
  // slabs are in flight; so are the traces of quadrilateral-face neighbours
  // outside this block (global memory, read-only during the stage)
  const real zM = M.w_mat[2 * Kp + e];
  int qnbr[3], qcode[3];
  real zPq[3];
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) {
    qnbr[ed] = M.w_nbr[(2 + ed) * Kp + e];
    qcode[ed] = M.w_code[(2 + ed) * Kp + e];
  }
  // (at N = 4 the traces held across the wait cost spills, and with the factor
  // computed in the stage they slow the factorising warp: there they are
  // requested after the wait, with the in-block ones)
  const bool early = N <= 3 && stored;
  Q4 nv[3][Nq];
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) {
    const int nbr = qnbr[ed];
    if (early && nbr >= 0 && (nbr >> 5) != blk) {
      const int ep = qcode[ed] >> 1, rev = qcode[ed] & 1;
      const real* base = qin + widx<N>(nbr >> 5, 0, nbr & 31);
#pragma unroll
      for (int m = 0; m < Nq; ++m) nv[ed][m] = ldg4(base, int64_t(j * Nt + O.tab.edge[ep][rev ? N - m : m]) * (kB * 4));
    }
  }
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) zPq[ed] = qnbr[ed] < 0 ? zM : M.w_mat[2 * Kp + qnbr[ed]];
  const int tnbr[2] = {M.w_nbr[0 * Kp + e], M.w_nbr[1 * Kp + e]};
  const int tcode[2] = {M.w_code[0 * Kp + e], M.w_code[1 * Kp + e]};
  real zPt[2];
#pragma unroll
  for (int fb = 0; fb < 2; ++fb)
    zPt[fb] = tnbr[fb] < 0 ? zM
                           : ((tcode[fb] & kCodeTet) ? M.t_mat[2 * M.Kt_pad + tnbr[fb]] : M.w_mat[2 * Kp + tnbr[fb]]);
  const bool src = M.nsrc > 0 && has_source(M, 6, e);
  // every lane of the geometry warp observes the coordinate copy itself
  bool geo_ok = true;
  __syncwarp();
  if (j == 0) {
    geo_ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[2], 0));
    if (geo_ok) wedge_geometry<G_STAGE>(sG, lane);
  }
  if (j == 1 && !stored) {
    // While the slabs are in flight: M^{tri,k} = sum_a J_a M_a with
    // J_a = A h_a / 2 (Lemma 3.1) from the vertices; L L^T factor row by row,
    // inverse diagonal stored in place of the diagonal.
    const int v0 = M.w_vid[0 * Kp + e], v1 = M.w_vid[1 * Kp + e], v2 = M.w_vid[2 * Kp + e];
    const int v3 = M.w_vid[3 * Kp + e], v4 = M.w_vid[4 * Kp + e], v5 = M.w_vid[5 * Kp + e];
    const real x0 = M.vx[v0], y0 = M.vy[v0];
    const real Ah = real(0.125) * ((M.vx[v1] - x0) * (M.vy[v2] - y0) - (M.vx[v2] - x0) * (M.vy[v1] - y0));
    const real J0 = Ah * (M.vz[v3] - M.vz[v0]), J1 = Ah * (M.vz[v4] - M.vz[v1]), J2 = Ah * (M.vz[v5] - M.vz[v2]);
#pragma unroll
    for (int i = 0; i < Nt; ++i) {
      real row[Nt];
#pragma unroll
      for (int l = 0; l < i; ++l) {
        real s = J0 * O.w.Ma[0][i * Nt + l] + J1 * O.w.Ma[1][i * Nt + l] + J2 * O.w.Ma[2][i * Nt + l];
#pragma unroll
        for (int k = 0; k < l; ++k) s -= row[k] * LQ(l * (l + 1) / 2 + k);
        row[l] = s * LQ(l * (l + 1) / 2 + l);
      }
      real d = J0 * O.w.Ma[0][i * Nt + i] + J1 * O.w.Ma[1][i * Nt + i] + J2 * O.w.Ma[2][i * Nt + i];
#pragma unroll
      for (int k = 0; k < i; ++k) d -= row[k] * row[k];
#pragma unroll
      for (int l = 0; l < i; ++l) LQ(i * (i + 1) / 2 + l) = row[l];
      LQ(i * (i + 1) / 2 + i) = rsqrt_r(d);
    }
  }
  if (leader) *status = (mbar_wait_bounded(&bar[0], 0) && geo_ok) ? 1 : 0;
  block_sync();
  if (*reinterpret_cast<volatile int*>(status) == 0) {
    // the state slab never arrived: report, let any copy in flight drain, leave
    if (leader) {
      atomicOr(M.err, kErrTimeout);
      if (res_early) mbar_wait_bounded(&bar[1], 0);
      mbar_wait_bounded(&bar[0], 0);
      mbar_wait_bounded(&bar[2], 0);
    }
    return;
  }

  // 1. prologue: quadrilateral-face fluxes of slice j applied straight into the
  //    weak-form accumulators (every warp); triangle-face fluxes (warps 0 and N)
  // accumulators of node i of the slice by field pairs: W01[i] = (p, u_x),
  // W23[i] = (u_y, u_z), so that the mass solve and the update run on packed pairs
  constexpr int NH = (Nt + 1) / 2;
  real2 W01[Nt], W23[Nt];
#pragma unroll
  for (int i = 0; i < Nt; ++i) W01[i] = W23[i] = dup2(real(0));
  // the neighbour node of triangle-face flux t of this warp (round-robin over
  // the warps, bottom then top): a tet's face node, or a wedge's bottom/top
  // node in this block's slab or in global memory; a boundary face reads its
  // own node.  With TF all are requested before the quadrilateral faces, whose
  // work covers the latency of the global ones.
  constexpr int NTT = (2 * Nt + Nq - 1) / Nq;
  auto tri_nbr_node = [&](int t) {
    const int idx = j + t * Nq;
    const int fb = idx >= Nt ? 1 : 0;
    const int k = idx - fb * Nt;
    const int nbr = tnbr[fb];
    const int code = tcode[fb];
    const bool bnd = nbr < 0;
    const bool ntet = !bnd && (code & kCodeTet) != 0;
    const int nf = bnd ? fb : (code >> 4) & 3;
    const int nk = bnd ? k : O.tab.tri_perm[code & 15][k];
    const int nbe = bnd ? e : nbr;
    const int node = ntet ? O.tab.tet_face[nf][nk] : (nf ? N * Nt : 0) + nk;
    const bool inblk = !ntet && (nbe >> 5) == blk;
    // explicit shared or global loads (a generic load would wait on the long scoreboard either way)
    return inblk ? lds4(sq, node, nbe & 31)
                 : ldg4(qin, ntet ? tidx<N>(M.tet_off, nbe >> 5, node, nbe & 31) : widx<N>(nbe >> 5, node, nbe & 31));
  };
  Q4 tnv[TF ? NTT : 1];
  if constexpr (TF) {
#pragma unroll
    for (int t = 0; t < NTT; ++t)
      if (j + t * Nq < 2 * Nt) tnv[t] = tri_nbr_node(t);
  }
  // N = 4 without TF: every triangle-face neighbour node is in shared memory
  // or a boundary ghost, and those fluxes go first, giving the quadrilateral
  // traces (read from global memory after the slab wait at this order) time to
  // arrive: 810 -> 778 us per stage on 524,288 wedges (at N = 3, whose
  // quadrilateral traces are requested before the wait, it measured 3.6% slower)
  constexpr bool tri_first = !TF && N == 4;
  if constexpr (tri_first) {
  // triangle-face node fluxes (bottom then top), spread round-robin over the warps
#pragma unroll
  for (int t = 0; t < NTT; ++t) {
    const int idx = j + t * Nq;
    if (idx >= 2 * Nt) break;
    const int fb = idx >= Nt ? 1 : 0;
    const int k = idx - fb * Nt;
    const real nn0 = GEO(fb ? G_NT0 : G_NB0), nn1 = GEO(fb ? G_NT1 : G_NB1), nn2 = GEO(fb ? G_NT2 : G_NB2);
    const int nbr = tnbr[fb];
    const Q4 o = lds4(sq, (fb ? N * Nt : 0) + k, lane);
    const real unM = fmar(nn2, o.w, fmar(nn1, o.v, nn0 * o.u));
    real tau_p, tau_u, bdp, bdun;
    taus(A.flux, zM, fb ? zPt[1] : zPt[0], tau_p, tau_u);
    boundary_jumps(A.bc, o.p, unM, bdp, bdun);
    const bool bnd = nbr < 0;
    Q4 nv;
    if constexpr (TF) nv = tnv[t];
    else nv = tri_nbr_node(t);
    // (explicit FMAs: both variants of the neighbour load give the same bits)
    const real dp = bnd ? bdp : nv.p - o.p;
    const real dun = bnd ? bdun : fmar(nn2, nv.w, fmar(nn1, nv.v, nn0 * nv.u)) - unM;
    real Fp, Fu;
    penalty_flux(dp, dun, tau_p, tau_u, Fp, Fu);
    sF[((2 * fb + 0) * Nt + k) * kB + lane] = Fp;
    sF[((2 * fb + 1) * Nt + k) * kB + lane] = Fu;
  }
  }
  // neighbour traces of quadrilateral faces whose neighbour lies in this block
  // (or, on a boundary face, the element's own trace, which the ghost state
  // then replaces) from the shared slab; the others were requested above (or,
  // at N = 4, now, from global memory)
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) {
    const int nbr = qnbr[ed];
    const bool bnd = nbr < 0;
    const bool inblk = bnd || (nbr >> 5) == blk;
    const int ep = bnd ? ed : qcode[ed] >> 1, rev = bnd ? 0 : qcode[ed] & 1;
    if (inblk) {
      const int nl = bnd ? lane : (nbr & 31);
#pragma unroll
      for (int m = 0; m < Nq; ++m) nv[ed][m] = lds4(sq, j * Nt + O.tab.edge[ep][rev ? N - m : m], nl);
    } else if (!early) {
      const real* base = qin + widx<N>(nbr >> 5, 0, nbr & 31);
#pragma unroll
      for (int m = 0; m < Nq; ++m) nv[ed][m] = ldg4(base, int64_t(j * Nt + O.tab.edge[ep][rev ? N - m : m]) * (kB * 4));
    }
  }
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) {
    const real nx = GEO(G_QNX0 + ed), ny = GEO(G_QNY0 + ed);
    real Fp[Nq], Fu[Nq];
    real tau_p, tau_u;
    taus(A.flux, zM, zPq[ed], tau_p, tau_u);
#pragma unroll
    for (int m = 0; m < Nq; ++m) {
      const Q4 o = lds4(sq, j * Nt + edge_node(N, ed, m), lane);
      real bdp, bdun;
      boundary_jumps(A.bc, o.p, nx * o.u + ny * o.v, bdp, bdun);
      const bool bnd = qnbr[ed] < 0;
      const real dp = bnd ? bdp : nv[ed][m].p - o.p;
      const real dun = bnd ? bdun : nx * (nv[ed][m].u - o.u) + ny * (nv[ed][m].v - o.v);
      penalty_flux(dp, dun, tau_p, tau_u, Fp[m], Fu[m]);
    }
    // W += M~_e F, M~_e = (L_e/4)(h_a Mea + h_b Meb) along the edge, identity in t
    // (Mea, Meb applied by output pairs: packed multiply-adds)
    const real ca = GEO(G_QCA0 + ed), cbq = GEO(G_QCB0 + ed);
    constexpr int NQH = (Nq + 1) / 2;
    real2 gpa[NQH], gpb[NQH], gua[NQH], gub[NQH];
#pragma unroll
    for (int h = 0; h < NQH; ++h) gpa[h] = gpb[h] = gua[h] = gub[h] = dup2(real(0));
#pragma unroll
    for (int n = 0; n < Nq; ++n) {
      const real2 fp2 = dup2(Fp[n]), fu2 = dup2(Fu[n]);
#pragma unroll
      for (int h = 0; h < NQH; ++h) {
        const real2 ea = cpair(O.w.MeaP, Nq, h, n), eb = cpair(O.w.MebP, Nq, h, n);
        gpa[h] = fma2(ea, fp2, gpa[h]);
        gpb[h] = fma2(eb, fp2, gpb[h]);
        gua[h] = fma2(ea, fu2, gua[h]);
        gub[h] = fma2(eb, fu2, gub[h]);
      }
    }
#pragma unroll
    for (int m = 0; m < Nq; ++m) {
      const bool hi = m & 1;
      const real2 pa = gpa[m >> 1], pb = gpb[m >> 1], ua = gua[m >> 1], ub = gub[m >> 1];
      const real gp = ca * (hi ? pa.y : pa.x) + cbq * (hi ? pb.y : pb.x);
      const real gu = ca * (hi ? ua.y : ua.x) + cbq * (hi ? ub.y : ub.x);
      const int i = edge_node(N, ed, m);
      W01[i].x += gp;
      W01[i].y += nx * gu;
      W23[i].x += ny * gu;
    }
  }
  if constexpr (!tri_first) {
  // triangle-face node fluxes (bottom then top), spread round-robin over the warps
#pragma unroll
  for (int t = 0; t < NTT; ++t) {
    const int idx = j + t * Nq;
    if (idx >= 2 * Nt) break;
    const int fb = idx >= Nt ? 1 : 0;
    const int k = idx - fb * Nt;
    const real nn0 = GEO(fb ? G_NT0 : G_NB0), nn1 = GEO(fb ? G_NT1 : G_NB1), nn2 = GEO(fb ? G_NT2 : G_NB2);
    const int nbr = tnbr[fb];
    const Q4 o = lds4(sq, (fb ? N * Nt : 0) + k, lane);
    const real unM = fmar(nn2, o.w, fmar(nn1, o.v, nn0 * o.u));
    real tau_p, tau_u, bdp, bdun;
    taus(A.flux, zM, fb ? zPt[1] : zPt[0], tau_p, tau_u);
    boundary_jumps(A.bc, o.p, unM, bdp, bdun);
    const bool bnd = nbr < 0;
    Q4 nv;
    if constexpr (TF) nv = tnv[t];
    else nv = tri_nbr_node(t);
    // (explicit FMAs: both variants of the neighbour load give the same bits)
    const real dp = bnd ? bdp : nv.p - o.p;
    const real dun = bnd ? bdun : fmar(nn2, nv.w, fmar(nn1, nv.v, nn0 * nv.u)) - unM;
    real Fp, Fu;
    penalty_flux(dp, dun, tau_p, tau_u, Fp, Fu);
    sF[((2 * fb + 0) * Nt + k) * kB + lane] = Fp;
    sF[((2 * fb + 1) * Nt + k) * kB + lane] = Fu;
  }
  }
  block_sync();

  // 2. slice j of every element of the block
  const real kappa = M.w_mat[0 * Kp + e], irho = M.w_mat[1 * Kp + e];
  {
    real dtr[Nq];
#pragma unroll
    for (int m = 0; m < Nq; ++m) dtr[m] = O.w.Dt[j * Nq + m];
    const real tj = O.w.gll[j];
    const real txJ = GEO(G_TX0) + tj * GEO(G_TX1);
    const real tyJ = GEO(G_TY0) + tj * GEO(G_TY1);
    const real Aj = GEO(G_A);
    const real cb = GEO(G_JFB) * O.w.ell0[j];
    const real ct = GEO(G_JFT) * O.w.ellN[j];
    if constexpr (OP == kOpFFMA) {
    // (a) pressure: G = -(t_xJ D_t u_x + t_yJ D_t u_y + A D_t u_z) + lifts; W = M^tri G
    real dp[Nt];
    {
      real G[Nt];
#pragma unroll
      for (int i = 0; i < Nt; ++i) {
        // D_t of the four fields as two packed pairs (p, u_x) and (u_y, u_z)
        real2 dpu = dup2(real(0)), dvw = dup2(real(0));
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          const Q4 v = lds4(sq, m * Nt + i, lane);
          const real2 d2 = dup2(dtr[m]);
          dpu = fma2(d2, mk2(v.p, v.u), dpu);
          dvw = fma2(d2, mk2(v.v, v.w), dvw);
        }
        dp[i] = dpu.x;
        G[i] = cb * sF[(0 * Nt + i) * kB + lane] + ct * sF[(2 * Nt + i) * kB + lane] -
               (txJ * dpu.y + tyJ * dvw.x + Aj * dvw.y);
      }
      real2 acc[NH];
      apply_pairs<Nt, Nt>(O.w.MP, G, acc);
#pragma unroll
      for (int i = 0; i < Nt; ++i) W01[i].x += pair_row(acc, i);
    }
    // (b) velocity: G_c = -t_cJ D_t p + n_c lifts; W = M^tri G
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const real tc = (c == 0) ? txJ : (c == 1 ? tyJ : Aj);
      const real nbc = GEO(G_NB0 + c) * cb, ntc = GEO(G_NT0 + c) * ct;
      real G[Nt];
#pragma unroll
      for (int i = 0; i < Nt; ++i)
        G[i] = nbc * sF[(1 * Nt + i) * kB + lane] + ntc * sF[(3 * Nt + i) * kB + lane] - tc * dp[i];
      real2 acc[NH];
      apply_pairs<Nt, Nt>(O.w.MP, G, acc);
#pragma unroll
      for (int i = 0; i < Nt; ++i) {
        if (c == 0) W01[i].y += pair_row(acc, i);
        else if (c == 1) W23[i].x += pair_row(acc, i);
        else W23[i].y += pair_row(acc, i);
      }
    }
    } else {
      // (a, b) on the tensor cores: the four vectors G of every element of
      // the block go to this warp's tile (columns lane * 4 + field), M^tri G
      // is formed one 16 x 8 output tile at a time in place, and each lane
      // reads its element's four results back
      const real nb0 = GEO(G_NB0) * cb, nb1 = GEO(G_NB1) * cb, nb2 = GEO(G_NB2) * cb;
      const real nt0 = GEO(G_NT0) * ct, nt1 = GEO(G_NT1) * ct, nt2 = GEO(G_NT2) * ct;
#pragma unroll
      for (int i = 0; i < Nt; ++i) {
        real dpp = 0, dux = 0, duy = 0, duz = 0;
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          const Q4 v = lds4(sq, m * Nt + i, lane);
          dpp += dtr[m] * v.p;
          dux += dtr[m] * v.u;
          duy += dtr[m] * v.v;
          duz += dtr[m] * v.w;
        }
        const real fp = sF[(1 * Nt + i) * kB + lane], fq = sF[(3 * Nt + i) * kB + lane];
        const float4 gv = make_float4(
            cb * sF[(0 * Nt + i) * kB + lane] + ct * sF[(2 * Nt + i) * kB + lane] - (txJ * dux + tyJ * duy + Aj * duz),
            nb0 * fp + nt0 * fq - txJ * dpp, nb1 * fp + nt1 * fq - tyJ * dpp, nb2 * fp + nt2 * fq - Aj * dpp);
        *reinterpret_cast<float4*>(sT + tile_at(i, lane * 4)) = gv;
      }
      __syncwarp();
      {
        AFrag<OP> Am;
        afrag_load<Nt, OP>(O.w.M, lane, Am);
        const int g = lane >> 2, t = lane & 3;
#pragma unroll 2
        for (int nt = 0; nt < 16; ++nt) {
          BFrag<OP> Bf;
          bfrag_load<Nt, OP>(sT, nt * 8 + g, lane, Bf);
          float d[4] = {0.f, 0.f, 0.f, 0.f};
          op_mma<Nt, OP>(Am, Bf, d);
          if (g < Nt) *reinterpret_cast<float2*>(sT + tile_at(g, nt * 8 + 2 * t)) = make_float2(d[0], d[1]);
          if (g + 8 < Nt) *reinterpret_cast<float2*>(sT + tile_at(g + 8, nt * 8 + 2 * t)) = make_float2(d[2], d[3]);
        }
      }
      __syncwarp();
#pragma unroll
      for (int i = 0; i < Nt; ++i) {
        const float4 w = *reinterpret_cast<const float4*>(sT + tile_at(i, lane * 4));
        W01[i] = add2(W01[i], mk2(w.x, w.y));
        W23[i] = add2(W23[i], mk2(w.z, w.w));
      }
      if (res_async) {
        // every warp is done with its tile: the residual slab may now land in their space
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        block_sync();
        if (leader) {
          mbar_expect_tx(&bar[1], slab_bytes);
          bulk_g2s(sr, resg + int64_t(blk) * 4 * Np * kB, slab_bytes, &bar[1]);
        }
      }
    }
  }
  // (d) X = (M^{tri,k})^{-1} W: forward and backward substitution, 4
  // right-hand sides, both sweeping the packed factor row by row (the
  // backward one in column-update form), four entries per shared load
  {
    // row i of the factor, entries q = i (i + 1) / 2 + k, k = 0..i
    auto load_row = [&](int i, real (&Lr)[Nt]) {
      const int a0 = i * (i + 1) / 2;
#pragma unroll
      for (int c4 = a0 >> 2; c4 <= (a0 + i) >> 2; ++c4) {
        const Q4 v = ldop4(sL + (c4 * kB + lane) * 4);
        const real vv[4] = {v.p, v.u, v.v, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int k = c4 * 4 + q - a0;
          if (k >= 0 && k <= i) Lr[k] = vv[q];
        }
      }
    };
#pragma unroll
    for (int i = 0; i < Nt; ++i) {
      real Lr[Nt];
      load_row(i, Lr);
#pragma unroll
      for (int k = 0; k < i; ++k) {
        const real2 nl = dup2(-Lr[k]);
        W01[i] = fma2(nl, W01[k], W01[i]);
        W23[i] = fma2(nl, W23[k], W23[i]);
      }
      const real2 d = dup2(Lr[i]);
      W01[i] = mul2(W01[i], d);
      W23[i] = mul2(W23[i], d);
    }
#pragma unroll
    for (int i = Nt - 1; i >= 0; --i) {
      real Lr[Nt];
      load_row(i, Lr);
      const real2 d = dup2(Lr[i]);
      W01[i] = mul2(W01[i], d);
      W23[i] = mul2(W23[i], d);
#pragma unroll
      for (int k = 0; k < i; ++k) {
        const real2 nl = dup2(-Lr[k]);
        W01[k] = fma2(nl, W01[i], W01[k]);
        W23[k] = fma2(nl, W23[i], W23[k]);
      }
    }
  }
  // (e) strong r, s parts of slice j (constant metric terms, Lemma 3.1), on
  // the CUDA cores for every variant (on the tensor cores the results would
  // have to pass through shared memory back to the element's lane, which
  // measured slower than these FMAs with constant operands)
  {
    // (D_r, D_s applied by output pairs, node l of the slice at a time)
    const real rx = GEO(G_RX), ry = GEO(G_RY), sx = GEO(G_SX), sy = GEO(G_SY);
    real2 dv[NH], pr[NH], ps[NH];
#pragma unroll
    for (int h = 0; h < NH; ++h) dv[h] = pr[h] = ps[h] = dup2(real(0));
#pragma unroll
    for (int l = 0; l < Nt; ++l) {
      const Q4 v = lds4(sq, j * Nt + l, lane);
      const real2 p2 = dup2(v.p), a2 = dup2(rx * v.u + ry * v.v), b2 = dup2(sx * v.u + sy * v.v);
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const real2 r2 = cpair(O.w.DrP, Nt, h, l), s2 = cpair(O.w.DsP, Nt, h, l);
        dv[h] = fma2(r2, a2, dv[h]);
        dv[h] = fma2(s2, b2, dv[h]);
        pr[h] = fma2(r2, p2, pr[h]);
        ps[h] = fma2(s2, p2, ps[h]);
      }
    }
#pragma unroll
    for (int i = 0; i < Nt; ++i) {
      const bool hi = i & 1;
      const real dvi = hi ? dv[i >> 1].y : dv[i >> 1].x;
      const real pri = hi ? pr[i >> 1].y : pr[i >> 1].x, psi = hi ? ps[i >> 1].y : ps[i >> 1].x;
      W01[i].x -= dvi;
      W01[i].y -= rx * pri + sx * psi;
      W23[i].x -= ry * pri + sy * psi;
    }
  }
  // (f) fused low-storage Runge-Kutta update (or plain right-hand side)
  if (res_async && !mbar_wait_bounded(&bar[1], 0)) {
    if (lane == 0) atomicOr(M.err, kErrTimeout);
    mbar_wait_bounded(&bar[1], 0);
    return;
  }
  if (src) add_sources(M, 6, e, j * Nt, Np, *M.clock + A.c_stage * double(A.dt), W01);
  if (e < M.Kw) {
#pragma unroll
    for (int i = 0; i < Nt; ++i) {
      const int n = j * Nt + i;
      const int64_t g = widx<N>(blk, n, lane);
      const real2 r01 = mul2(W01[i], mk2(kappa, irho)), r23 = mul2(W23[i], dup2(irho));
      const Q4 r{r01.x, r01.y, r23.x, r23.y};
      if (rk) {
        // res = a res + dt r, q = g q + b res, on packed pairs
        const Q4 r0 = stage_res<N, OP>() ? lds4(sr, n, lane) : ld4(resg, g);
        const real2 a2 = dup2(A.rk_a), dt2 = dup2(A.dt), g2 = dup2(A.rk_g), b2 = dup2(A.rk_b);
        const real2 rr01 = fma2(a2, mk2(r0.p, r0.u), mul2(dt2, r01));
        const real2 rr23 = fma2(a2, mk2(r0.v, r0.w), mul2(dt2, r23));
        const Q4 q0 = lds4(sq, n, lane);
        const real2 q01 = fma2(g2, mk2(q0.p, q0.u), mul2(b2, rr01));
        const real2 q23 = fma2(g2, mk2(q0.v, q0.w), mul2(b2, rr23));
        st4(resg, g, Q4{rr01.x, rr01.y, rr23.x, rr23.y});
        st4(qout, g, Q4{q01.x, q01.y, q23.x, q23.y});
        if (A.rhs_out) st4(A.rhs_out, g, r);
      } else {
        st4(qout, g, r);
      }
    }
  }
#undef GEO
#undef LQ
}

// ---------------------------------------------------------------------------
// tet stage: one 32-tet block per CTA (lane = tet), 4 warps.  Bulk copies move
// the tet operators ([l][i] (D_r, D_s, D_t)(i, l) records and the lift, laid
// out per warp chunk), the block's vertex coordinates and its state slab into
// shared memory.  Every warp evaluates the affine geometry of the 32 tets;
// warp f forms the fluxes of face f into a shared table; warp w then forms
// the volume terms of output nodes [w C, w C + C) and, after one barrier,
// their lift and update.
// All warps run the same code.
// ---------------------------------------------------------------------------
template <int N>
__host__ __device__ constexpr int tet_chunk() {  // output nodes per warp
  return (npt_of(N) + 3) / 4;
}
template <int N>
__host__ __device__ constexpr int tet_chunk_pad() {  // lift record length per face node (multiple of 4)
  return (tet_chunk<N>() + 3) / 4 * 4;
}
template <int N>
__host__ __device__ constexpr int tet_ops_image_reals() {  // the global image t_ops: D records, then the lift
  return 4 * npt_of(N) * npt_of(N) + 4 * (4 * nt_of(N)) * tet_chunk_pad<N>();
}
// Whether the lift rows are copied to shared memory with the derivative
// records: everywhere but FP64 at N = 5, where the whole image would exceed a
// CTA's shared memory; there the warps read their lift rows (uniform
// addresses) from global memory.
template <int N>
__host__ __device__ constexpr bool tet_lift_smem() {
  return 128 + (tet_ops_image_reals<N>() + 4 * npt_of(N) * kB + 8 * nt_of(N) * kB + 12 * kB +
                ((sizeof(real) == 4 && N <= 3) ? 4 * npt_of(N) * kB : 0)) * int(sizeof(real)) <= 227 * 1024;
}
template <int N>
__host__ __device__ constexpr int tet_ops_reals() {  // the part of the image in shared memory
  return tet_lift_smem<N>() ? tet_ops_image_reals<N>() : 4 * npt_of(N) * npt_of(N);
}
// The residual slab is bulk-copied too where it costs no CTA per SM (FP32,
// N <= 3); elsewhere the update reads it from global memory.
template <int N>
__host__ __device__ constexpr bool tet_stage_res() {
  return sizeof(real) == 4 && N <= 3;
}
// 128-byte header (4 mbarriers), operators, slab [Np][32][4], fluxes
// [4 faces][2][Nt][32], vertex coordinates [12][32], residual slab [Np][32][4]
template <int N>
__host__ __device__ constexpr int tet_smem_reals() {
  return tet_ops_reals<N>() + 4 * npt_of(N) * kB + 8 * nt_of(N) * kB + 12 * kB +
         (tet_stage_res<N>() ? 4 * npt_of(N) * kB : 0);
}
template <int N>
__host__ __device__ constexpr int tet_smem_bytes() {
  return 128 + tet_smem_reals<N>() * int(sizeof(real));
}

template <int N>
__global__ void __launch_bounds__(128, (sizeof(REAL) == 4) ? (N >= 4 ? 3 : 5) : 2)
    k_tet_stage(const StageArgs<real> A, bool rk) {
  constexpr int Np = npt_of(N), Nt = nt_of(N), C = tet_chunk<N>(), CP = tet_chunk_pad<N>();
  const AllOps<N, real>& O = OPS<N>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);  // [0] operators, [1] coordinates, [2] state, [3] residual
  real* sOp = reinterpret_cast<real*>(smem_raw + 128);
  real* sL = sOp + 4 * Np * Np;  // lift [warp][4 Nt][CP]
  real* sq = sOp + tet_ops_reals<N>();
  real* sF = sq + 4 * Np * kB;
  real* sX = sF + 8 * Nt * kB;
  real* sr = sX + 12 * kB;  // residual slab (tet_stage_res)
  constexpr bool stage_res = tet_stage_res<N>();
  const DevMesh<real>& M = A.m;
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int blk = blockIdx.x;
  const int e = blk * kB + lane;
  const int Kp = M.Kt_pad;
  constexpr uint32_t slab_bytes = uint32_t(4 * Np * kB * sizeof(real)), xyz_bytes = uint32_t(12 * kB * sizeof(real));
  constexpr uint32_t ops_bytes = uint32_t(tet_ops_reals<N>() * sizeof(real));
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    mbar_init(&bar[3], 1);
    fence_mbar_init();
    mbar_expect_tx(&bar[1], xyz_bytes);
    bulk_g2s(sX, M.t_xyz + int64_t(blk) * 12 * kB, xyz_bytes, &bar[1]);
    mbar_expect_tx(&bar[2], slab_bytes);
    bulk_g2s(sq, A.q_in + M.tet_off + int64_t(blk) * 4 * Np * kB, slab_bytes, &bar[2]);
    mbar_expect_tx(&bar[0], ops_bytes);
    bulk_g2s(sOp, M.t_ops, ops_bytes, &bar[0]);
    if (stage_res && rk) {
      mbar_expect_tx(&bar[3], slab_bytes);
      bulk_g2s(sr, A.res + M.tet_off + int64_t(blk) * 4 * Np * kB, slab_bytes, &bar[3]);
    }
  }
  // face neighbours, impedances, material and the source flag while the copies fly
  const real kappa = M.t_mat[0 * Kp + e], irho = M.t_mat[1 * Kp + e], zM = M.t_mat[2 * Kp + e];
  int nbr = M.t_nbr[w * Kp + e], code = M.t_code[w * Kp + e];  // this warp's face w
  const real zP = nbr < 0 ? zM : ((code & kCodeTet) ? M.t_mat[2 * Kp + nbr] : M.w_mat[2 * M.Kw_pad + nbr]);
  const bool src = M.nsrc > 0 && has_source(M, 4, e);
  // out-of-block neighbour face nodes of this warp's face, requested before the waits
  Q4 nvs[Nt];
  const bool t_bnd = nbr < 0;
  const bool t_ntet = !t_bnd && (code & kCodeTet) != 0;
  const int t_nbe = t_bnd ? e : nbr;
  const bool t_inblk = t_bnd || (t_ntet && (t_nbe >> 5) == blk);
  if (!t_inblk) {
    const int nfc = (code >> 4) & 3, perm = code & 15;
    const real* nb = A.q_in + (t_ntet ? tidx<N>(M.tet_off, t_nbe >> 5, 0, t_nbe & 31) : widx<N>(t_nbe >> 5, 0, t_nbe & 31));
#pragma unroll
    for (int k = 0; k < Nt; ++k) {
      const int nk = O.tab.tri_perm[perm][k];
      nvs[k] = ldg4(nb, int64_t(t_ntet ? O.tab.tet_face[nfc][nk] : (nfc ? N * Nt : 0) + nk) * (kB * 4));
    }
  }
  __syncthreads();  // the mbarriers are initialised

  // affine geometry: x = sum_v lambda_v X_v on the bi-unit reference tet
  bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[1], 0));
  real Ri[3][3], nf[4][3], sJ[4];  // d r_m / d x_d, outward unit normals, J_f / J
  {
    real X[4][3];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int d = 0; d < 3; ++d) X[v][d] = sX[(v * 3 + d) * kB + lane];
    real G[3][3];  // G[d][m] = d x_d / d r_m
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int m = 0; m < 3; ++m) G[d][m] = real(0.5) * (X[m + 1][d] - X[0][d]);
    const real J = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
                   G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) + G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
    const real iJ = real(1) / J;
    Ri[0][0] = (G[1][1] * G[2][2] - G[1][2] * G[2][1]) * iJ;
    Ri[0][1] = (G[0][2] * G[2][1] - G[0][1] * G[2][2]) * iJ;
    Ri[0][2] = (G[0][1] * G[1][2] - G[0][2] * G[1][1]) * iJ;
    Ri[1][0] = (G[1][2] * G[2][0] - G[1][0] * G[2][2]) * iJ;
    Ri[1][1] = (G[0][0] * G[2][2] - G[0][2] * G[2][0]) * iJ;
    Ri[1][2] = (G[0][2] * G[1][0] - G[0][0] * G[1][2]) * iJ;
    Ri[2][0] = (G[1][0] * G[2][1] - G[1][1] * G[2][0]) * iJ;
    Ri[2][1] = (G[0][1] * G[2][0] - G[0][0] * G[2][1]) * iJ;
    Ri[2][2] = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) * iJ;
    constexpr int fv[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};
    constexpr int fo[4] = {3, 2, 0, 1};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const real ax = X[fv[f][1]][0] - X[fv[f][0]][0], ay = X[fv[f][1]][1] - X[fv[f][0]][1],
                 az = X[fv[f][1]][2] - X[fv[f][0]][2];
      const real bx = X[fv[f][2]][0] - X[fv[f][0]][0], by = X[fv[f][2]][1] - X[fv[f][0]][1],
                 bz = X[fv[f][2]][2] - X[fv[f][0]][2];
      const real cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
      const real cc = cx * cx + cy * cy + cz * cz, ic = rsqrt_r(cc);
      const real ox = X[fo[f]][0] - X[fv[f][0]][0], oy = X[fo[f]][1] - X[fv[f][0]][1], oz = X[fo[f]][2] - X[fv[f][0]][2];
      const real sgn = (cx * ox + cy * oy + cz * oz > 0) ? real(-1) : real(1);  // away from the opposite vertex
      nf[f][0] = sgn * cx * ic;
      nf[f][1] = sgn * cy * ic;
      nf[f][2] = sgn * cz * ic;
      sJ[f] = real(0.25) * cc * ic * iJ;
    }
  }
  ok = ok && __all_sync(0xffffffffu, mbar_wait_bounded(&bar[2], 0));
  if (!ok) {
    // a copy never arrived: report, let the copies in flight drain, leave
    if (threadIdx.x == 0) atomicOr(M.err, kErrTimeout);
    if (lane == 0) {
      mbar_wait_bounded(&bar[0], 0);
      mbar_wait_bounded(&bar[1], 0);
      mbar_wait_bounded(&bar[2], 0);
      if (stage_res && rk) mbar_wait_bounded(&bar[3], 0);
    }
    return;
  }

  // fluxes of face w, scaled by J_f / J, into the shared flux table
  {
    const int f = w;
    real n0 = nf[0][0], n1 = nf[0][1], n2 = nf[0][2], sj = sJ[0];
#pragma unroll
    for (int g = 1; g < 4; ++g)
      if (f == g) {
        n0 = nf[g][0];
        n1 = nf[g][1];
        n2 = nf[g][2];
        sj = sJ[g];
      }
    real tau_p, tau_u;
    taus(A.flux, zM, zP, tau_p, tau_u);
    const bool bnd = nbr < 0;
    const bool ntet = !bnd && (code & kCodeTet) != 0;
    const int nfc = (code >> 4) & 3, perm = code & 15;
    const int nbe = bnd ? e : nbr;
    const bool inblk = bnd || (ntet && (nbe >> 5) == blk);
    // the neighbour's face nodes, all requested at once: this block's own slab
    // (shared loads), or another tet block's or a wedge block's in global memory
    if (inblk) {
#pragma unroll
      for (int k = 0; k < Nt; ++k) {
        const int nk = bnd ? k : O.tab.tri_perm[perm][k];
        nvs[k] = lds4(sq, bnd ? O.tab.tet_face[f][k] : O.tab.tet_face[nfc][nk], nbe & 31);
      }
    }
#pragma unroll
    for (int k = 0; k < Nt; ++k) {
      const int own = O.tab.tet_face[f][k];
      const Q4 o = lds4(sq, own, lane);
      const real unM = n0 * o.u + n1 * o.v + n2 * o.w;
      const Q4 nv = nvs[k];
      real bdp, bdun;
      boundary_jumps(A.bc, o.p, unM, bdp, bdun);
      const real dp = bnd ? bdp : nv.p - o.p;
      const real dun = bnd ? bdun : n0 * nv.u + n1 * nv.v + n2 * nv.w - unM;
      real Fp, Fu;
      penalty_flux(dp, dun, tau_p, tau_u, Fp, Fu);
      sF[((f * 2 + 0) * Nt + k) * kB + lane] = sj * Fp;
      sF[((f * 2 + 1) * Nt + k) * kB + lane] = sj * Fu;
    }
  }
  if (!__all_sync(0xffffffffu, mbar_wait_bounded(&bar[0], 0)) && lane == 0) atomicOr(M.err, kErrTimeout);

  // output nodes [I0, I0 + C) of this warp: volume terms (the slab and the
  // operators only), then, once every warp's face fluxes are in the table,
  // the lift and the update
  const int I0 = w * C;
  // results of the warp's outputs by output pairs (c, c + 1): ap2 the pressure,
  // au2[d] the velocity components (packed multiply-adds)
  constexpr int CH = (C + 1) / 2;
  real2 ap2[CH], au2[3][CH];
  {
    // per output: (D_r p, D_s p) and D_t p; (D_r w_r + D_t w_t, D_s w_s) with
    // w = the reference-direction velocity components
    real2 drs[C], sab[C];
    real dt[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      drs[c] = sab[c] = dup2(real(0));
      dt[c] = real(0);
    }
    const real* opI = sOp + I0 * 4;  // records (l, I0 + c) at opI + (l Np + c) 4
#pragma unroll 4
    for (int l = 0; l < Np; ++l) {
      const Q4 v = lds4(sq, l, lane);
      const real wr = Ri[0][0] * v.u + Ri[0][1] * v.v + Ri[0][2] * v.w;
      const real ws = Ri[1][0] * v.u + Ri[1][1] * v.v + Ri[1][2] * v.w;
      const real wt = Ri[2][0] * v.u + Ri[2][1] * v.v + Ri[2][2] * v.w;
      const real2 pp = dup2(v.p), wrs = mk2(wr, ws);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const Q4 d = ldop4(opI + (l * Np + c) * 4);  // I0 + c >= Np: unused records, results dropped
        const real2 dpu = mk2(d.p, d.u);
        drs[c] = fma2(dpu, pp, drs[c]);
        dt[c] += d.v * v.p;
        sab[c] = fma2(dpu, wrs, sab[c]);
        sab[c].x += d.v * wt;
      }
    }
#pragma unroll
    for (int h = 0; h < CH; ++h) {
      const int c0 = 2 * h, c1 = 2 * h + 1 < C ? 2 * h + 1 : 2 * h;
      ap2[h] = mk2(-(sab[c0].x + sab[c0].y), -(sab[c1].x + sab[c1].y));
#pragma unroll
      for (int d = 0; d < 3; ++d)
        au2[d][h] = mk2(-(Ri[0][d] * drs[c0].x + Ri[1][d] * drs[c0].y + Ri[2][d] * dt[c0]),
                        -(Ri[0][d] * drs[c1].x + Ri[1][d] * drs[c1].y + Ri[2][d] * dt[c1]));
    }
  }
  __syncthreads();
  {
    // this warp's lift records [4 Nt][CP] (shared memory, or the global image)
    const real* lw = (tet_lift_smem<N>() ? sL : M.t_ops + 4 * Np * Np) + w * (4 * Nt) * CP;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      real2 lu2[CH];
#pragma unroll
      for (int h = 0; h < CH; ++h) lu2[h] = dup2(real(0));
#pragma unroll 5
      for (int k = 0; k < Nt; ++k) {
        const real2 fp2 = dup2(sF[((f * 2 + 0) * Nt + k) * kB + lane]);
        const real2 fu2 = dup2(sF[((f * 2 + 1) * Nt + k) * kB + lane]);
#pragma unroll
        for (int c4 = 0; c4 < CP; c4 += 4) {
          const Q4 L = ldop4(lw + (f * Nt + k) * CP + c4);
          const real2 La = mk2(L.p, L.u), Lb = mk2(L.v, L.w);
          const int h = c4 / 2;
          if (h < CH) {
            ap2[h] = fma2(La, fp2, ap2[h]);
            lu2[h] = fma2(La, fu2, lu2[h]);
          }
          if (h + 1 < CH) {
            ap2[h + 1] = fma2(Lb, fp2, ap2[h + 1]);
            lu2[h + 1] = fma2(Lb, fu2, lu2[h + 1]);
          }
        }
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const real2 n2 = dup2(nf[f][d]);
#pragma unroll
        for (int h = 0; h < CH; ++h) au2[d][h] = fma2(n2, lu2[h], au2[d][h]);
      }
    }
  }
  real ap[C];
#pragma unroll
  for (int c = 0; c < C; ++c) ap[c] = pair_row(ap2, c);
  if (src) add_sources(M, 4, e, I0, Np, *M.clock + A.c_stage * double(A.dt), ap);
  if (stage_res && rk && !__all_sync(0xffffffffu, mbar_wait_bounded(&bar[3], 0))) {
    // the residual slab never arrived: report, let the copy drain, leave
    if (lane == 0) {
      atomicOr(M.err, kErrTimeout);
      mbar_wait_bounded(&bar[3], 0);
    }
    return;
  }
  if (e < M.Kt) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      if (I0 + c < Np) {
        const int i = I0 + c;
        const int64_t gi = tidx<N>(M.tet_off, blk, i, lane);
        const real2 r01 = mul2(mk2(ap[c], pair_row(au2[0], c)), mk2(kappa, irho));
        const real2 r23 = mul2(mk2(pair_row(au2[1], c), pair_row(au2[2], c)), dup2(irho));
        const Q4 r{r01.x, r01.y, r23.x, r23.y};
        if (rk) {
          // res = a res + dt r, q = g q + b res, on packed pairs
          const Q4 r0 = stage_res ? lds4(sr, i, lane) : ld4(A.res, gi);
          const real2 a2 = dup2(A.rk_a), dt2 = dup2(A.dt), g2 = dup2(A.rk_g), b2 = dup2(A.rk_b);
          const real2 rr01 = fma2(a2, mk2(r0.p, r0.u), mul2(dt2, r01));
          const real2 rr23 = fma2(a2, mk2(r0.v, r0.w), mul2(dt2, r23));
          const Q4 q0 = lds4(sq, i, lane);
          const real2 q01 = fma2(g2, mk2(q0.p, q0.u), mul2(b2, rr01));
          const real2 q23 = fma2(g2, mk2(q0.v, q0.w), mul2(b2, rr23));
          st4(A.res, gi, Q4{rr01.x, rr01.y, rr23.x, rr23.y});
          st4(A.q_out, gi, Q4{q01.x, q01.y, q23.x, q23.y});
          if (A.rhs_out) st4(A.rhs_out, gi, r);
        } else {
          st4(A.q_out, gi, r);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// canonical <-> packed layout
// ---------------------------------------------------------------------------
// Canonical [shot][field][node] <-> packed [block][node][lane][field] layout.
// One CTA per 32-element block at a time: the block's values pass through a
// [field][node][lane] shared tile (lane pitch 33, so neither phase has bank
// conflicts), the canonical side is read or written one element's contiguous
// node run at a time and the packed side in 16-byte [node][lane] records.
// Padding lanes (e >= K) are neither read nor written.
template <int N>
__host__ __device__ constexpr int pack_smem_bytes() {
  return 4 * npw_of(N) * 33 * int(sizeof(real));
}

template <int N>
__global__ void __launch_bounds__(256) k_pack(const DevMesh<real> M, const real* __restrict__ canon,
                                              real* __restrict__ packed, bool unpack) {
  constexpr int Npw = npw_of(N), Npt = npt_of(N);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  real* tile = reinterpret_cast<real*>(smem_raw);  // [4][Np][33]
  real* cw = const_cast<real*>(canon);
  const int64_t T = M.total_nodes;
  for (int b = blockIdx.x; b < M.nblk_w + M.nblk_t; b += gridDim.x) {
    const bool tet = b >= M.nblk_w;
    const int blk = tet ? b - M.nblk_w : b;
    const int Np = tet ? Npt : Npw, K = tet ? M.Kt : M.Kw;
    const int64_t* cmap = tet ? M.t_canon : M.w_canon;
    real* pk = packed + (tet ? tidx<N>(M.tet_off, blk, 0, 0) : widx<N>(blk, 0, 0));
    const int items = Np * kB;
    if (!unpack) {
      for (int t = threadIdx.x; t < items; t += blockDim.x) {
        const int l = t / Np, n = t - l * Np, e = blk * kB + l;
        if (e < K) {
          const int64_t c = cmap[e] + n;
#pragma unroll
          for (int f = 0; f < 4; ++f) tile[(f * Np + n) * 33 + l] = canon[f * T + c];
        }
      }
      __syncthreads();
      for (int t = threadIdx.x; t < items; t += blockDim.x) {
        const int l = t & 31, n = t >> 5;
        if (blk * kB + l < K)
          st4(pk, int64_t(t) * 4,
              Q4{tile[(0 * Np + n) * 33 + l], tile[(1 * Np + n) * 33 + l], tile[(2 * Np + n) * 33 + l],
                 tile[(3 * Np + n) * 33 + l]});
      }
    } else {
      for (int t = threadIdx.x; t < items; t += blockDim.x) {
        const int l = t & 31, n = t >> 5;
        if (blk * kB + l < K) {
          const Q4 v = ld4(pk, int64_t(t) * 4);
          tile[(0 * Np + n) * 33 + l] = v.p;
          tile[(1 * Np + n) * 33 + l] = v.u;
          tile[(2 * Np + n) * 33 + l] = v.v;
          tile[(3 * Np + n) * 33 + l] = v.w;
        }
      }
      __syncthreads();
      for (int t = threadIdx.x; t < items; t += blockDim.x) {
        const int l = t / Np, n = t - l * Np, e = blk * kB + l;
        if (e < K) {
          const int64_t c = cmap[e] + n;
#pragma unroll
          for (int f = 0; f < 4; ++f) cw[f * T + c] = tile[(f * Np + n) * 33 + l];
        }
      }
    }
    __syncthreads();  // the tile is reused by the next block
  }
}

// ---------------------------------------------------------------------------
// discrete energy (Section 4.1), double accumulation, deterministic order
// ---------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(128) k_energy(const DevMesh<real> M, const real* __restrict__ q) {
  constexpr int Nt = nt_of(N), Nq = N + 1, Npw = npw_of(N), Npt = npt_of(N);
  const AllOps<N, real>& O = OPS<N>();
  const int nblk_cta_w = (M.nblk_w + 3) / 4;
  double E = 0.0;
  const int gw = blockIdx.x * 4 + (threadIdx.x >> 5);  // 32-element block handled by this warp
  const int lane = threadIdx.x & 31;
  if (blockIdx.x < nblk_cta_w) {
    const int e = gw * kB + lane;
    if (gw < M.nblk_w && e < M.Kw) {
      const int Kp = M.Kw_pad;
      const int vb0 = M.w_vid[0 * Kp + e], vb1 = M.w_vid[1 * Kp + e], vb2 = M.w_vid[2 * Kp + e];
      const double x0 = M.vx[vb0], x1 = M.vx[vb1], x2 = M.vx[vb2];
      const double y0 = M.vy[vb0], y1 = M.vy[vb1], y2 = M.vy[vb2];
      const double A = 0.25 * ((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0));
      double Ja[3];
      for (int a = 0; a < 3; ++a) Ja[a] = 0.5 * A * (double(M.vz[M.w_vid[(3 + a) * Kp + e]]) - double(M.vz[M.w_vid[a * Kp + e]]));
      const double wgt[4] = {1.0 / double(M.w_mat[0 * Kp + e]), 1.0 / double(M.w_mat[1 * Kp + e]),
                             1.0 / double(M.w_mat[1 * Kp + e]), 1.0 / double(M.w_mat[1 * Kp + e])};
#pragma unroll 1
      for (int f = 0; f < 4; ++f) {
        double ef = 0.0;
#pragma unroll 1
        for (int jp = 0; jp < Nq; ++jp)
#pragma unroll 1
          for (int jj = 0; jj < Nq; ++jj) {
            const double m1 = double(O.w.M1[jj * Nq + jp]);
            double d = 0.0;
#pragma unroll 1
            for (int i = 0; i < Nt; ++i) {
              double s = 0.0;
#pragma unroll 1
              for (int l = 0; l < Nt; ++l) {
                const double mt = Ja[0] * double(O.w.Ma[0][i * Nt + l]) + Ja[1] * double(O.w.Ma[1][i * Nt + l]) +
                                  Ja[2] * double(O.w.Ma[2][i * Nt + l]);
                s += mt * double(q[widx<N>(gw, jp * Nt + l, lane) + f]);
              }
              d += double(q[widx<N>(gw, jj * Nt + i, lane) + f]) * s;
            }
            ef += m1 * d;
          }
        E += wgt[f] * ef;
      }
    }
  } else {
    const int gt = gw - nblk_cta_w * 4;
    const int e = gt * kB + lane;
    if (gt < M.nblk_t && e < M.Kt) {
      const int Kp = M.Kt_pad;
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
      const double wgt[4] = {1.0 / double(M.t_mat[0 * Kp + e]), 1.0 / double(M.t_mat[1 * Kp + e]),
                             1.0 / double(M.t_mat[1 * Kp + e]), 1.0 / double(M.t_mat[1 * Kp + e])};
#pragma unroll 1
      for (int f = 0; f < 4; ++f) {
        double ef = 0.0;
#pragma unroll 1
        for (int i = 0; i < Npt; ++i) {
          double s = 0.0;
#pragma unroll 1
          for (int l = 0; l < Npt; ++l) s += double(M.tet_mass[i * Npt + l]) * double(q[tidx<N>(M.tet_off, gt, l, lane) + f]);
          ef += s * double(q[tidx<N>(M.tet_off, gt, i, lane) + f]);
        }
        E += wgt[f] * J * ef;
      }
    }
  }
  // block reduction in a fixed order
  __shared__ double red[128];
  red[threadIdx.x] = E;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) M.partials[blockIdx.x] = 0.5 * red[0];
  (void)Npw;
}

__global__ void k_energy_final(const double* __restrict__ partials, int n, double* out, int* err) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partials[i];
    *out = s;
    if (!isfinite(s)) atomicOr(err, kErrNonfinite);
  }
}

}  // namespace REALNS
}  // namespace dgw

#include "adjoint_kernels.cuh"
#include "stage_split.cuh"

namespace dgw {
namespace REALNS {


// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// one-time per device: opt in to the dynamic shared memory the stages use
template <int N, int OP>
cudaError_t prepare_op() {
  return cudaFuncSetAttribute(k_wedge_stage<N, 1, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              wedge_smem_bytes<N, 1, OP>());
}
template <int N>
int prepare_n() {
  constexpr int b2 = wedge_bpc_onthefly<N>();
  cudaError_t err = cudaFuncSetAttribute(k_wedge_stage<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         wedge_smem_bytes<N, 1>());
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_wedge_stage<N, 1, kOpFFMA, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               wedge_smem_bytes<N, 1>());
  if constexpr (sizeof(real) == 4) {
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_wedge_stage_split<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 split_smem_bytes<N>());
    if constexpr (nt_of(N) <= 16) {  // one 16-row tile holds a slice: tensor-core applies
      if (err == cudaSuccess) err = prepare_op<N, kOpTF32x3>();
      if (err == cudaSuccess) err = prepare_op<N, kOpTF32>();
      if (err == cudaSuccess) err = prepare_op<N, kOpBF16>();
    }
  }
  if (err == cudaSuccess && b2 != 1)
    err = cudaFuncSetAttribute(k_wedge_stage<N, b2, kOpFFMA, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               wedge_smem_bytes<N, b2>());
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_tet_stage<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, tet_smem_bytes<N>());
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_pack<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, pack_smem_bytes<N>());
  // the gradient kernels where their shared memory fits one CTA (not FP64 at N = 5,
  // whose adjoint the library refuses)
  if constexpr (grad_smem_bytes<N>() <= 227 * 1024) {
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_wedge_grad<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 grad_smem_bytes<N>());
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_wedge_grad<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 grad_smem_bytes<N>());
  }
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute(k_tet_grad<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, tgrad_smem_bytes<N>());
  return int(err);
}

template <int N, int OP>
void launch_op(const StageArgs<real>& a, bool rk, cudaStream_t s) {
  k_wedge_stage<N, 1, OP><<<a.m.nblk_w, 32 * (N + 1), wedge_smem_bytes<N, 1, OP>(), s>>>(a, rk);
}
template <int N>
int launch_stage_n(const StageArgs<real>& a, bool rk, cudaStream_t s, cudaStream_t st, cudaEvent_t ev_fork,
                   cudaEvent_t ev_join) {
  // wedges and tets of one stage are independent (each reads the stage input,
  // writes only its own elements): with a second stream the tet stage runs on
  // it, forked from and joined back into s (also inside a graph capture), so
  // the two kernels share the GPU instead of running back to back
  const bool fork = a.m.nblk_w > 0 && a.m.nblk_t > 0 && st != nullptr && ev_fork != nullptr && ev_join != nullptr;
  if (fork) {
    cudaError_t err = cudaEventRecord(ev_fork, s);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(st, ev_fork, 0);
    if (err != cudaSuccess) return int(err);
    k_tet_stage<N><<<a.m.nblk_t, 128, tet_smem_bytes<N>(), st>>>(a, rk);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(ev_join, st);
    if (err != cudaSuccess) return int(err);
  }
  if (a.m.nblk_w > 0) {
    constexpr int b2 = wedge_bpc_onthefly<N>();
    const int want = a.wedge_bpc > 0 ? a.wedge_bpc : (a.m.w_fac != nullptr ? 1 : b2);
    bool done = false;
    if constexpr (sizeof(real) == 4) {
      // the field-pair split kernel (FP32 CUDA-core applies, stored mass
      // factor): when the autotuner or dg_set_launch_variant chose it
      const bool split = a.op == kOpFFMA && a.m.w_fac != nullptr && a.split > 0;
      if (split) {
        k_wedge_stage_split<N><<<a.m.nblk_w, 64 * (N + 1), split_smem_bytes<N>(), s>>>(a, rk);
        done = true;
      }
    }
    if constexpr (sizeof(real) == 4 && nt_of(N) <= 16) {
      done = done || a.op != kOpFFMA;
      if (a.op == kOpTF32x3) launch_op<N, kOpTF32x3>(a, rk, s);
      else if (a.op == kOpTF32) launch_op<N, kOpTF32>(a, rk, s);
      else if (a.op == kOpBF16) launch_op<N, kOpBF16>(a, rk, s);
    }
    if (done) {
    } else if ((want == 1 || b2 == 1) && a.tri_far)
      k_wedge_stage<N, 1, kOpFFMA, true><<<a.m.nblk_w, 32 * (N + 1), wedge_smem_bytes<N, 1>(), s>>>(a, rk);
    else if (want == 1 || b2 == 1)
      k_wedge_stage<N, 1><<<a.m.nblk_w, 32 * (N + 1), wedge_smem_bytes<N, 1>(), s>>>(a, rk);
    else  // (two blocks per CTA: the early triangle-face requests measured 402 -> 371 us on 524,288 wedges)
      k_wedge_stage<N, b2, kOpFFMA, true><<<(a.m.nblk_w + b2 - 1) / b2, 32 * (N + 1) * b2, wedge_smem_bytes<N, b2>(),
                                            s>>>(a, rk);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return int(err);
  }
  if (fork) return int(cudaStreamWaitEvent(s, ev_join, 0));
  if (a.m.nblk_t > 0) {
    k_tet_stage<N><<<a.m.nblk_t, 128, tet_smem_bytes<N>(), s>>>(a, rk);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return int(err);
  }
  return 0;
}

template <int N>
int launch_pack_n(const DevMesh<real>& m, const real* canon, real* packed, bool unpack, cudaStream_t s) {
  int blocks = m.nblk_w + m.nblk_t;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  k_pack<N><<<blocks, 256, pack_smem_bytes<N>(), s>>>(m, canon, packed, unpack);
  return int(cudaGetLastError());
}

template <int N>
int launch_energy_n(const DevMesh<real>& m, const real* q, cudaStream_t s) {
  const int nw = (m.nblk_w + 3) / 4, nt = (m.nblk_t + 3) / 4;
  const int grid = nw + nt;
  if (grid > 0) k_energy<N><<<grid, 128, 0, s>>>(m, q);
  k_energy_final<<<1, 32, 0, s>>>(m.partials, grid, m.energy, m.err);
  return int(cudaGetLastError());
}

}  // namespace REALNS
}  // namespace dgw

// extern launchers of this translation unit (order NORD, precision REAL)
#define DGW_CAT2(a, b) a##b
#define DGW_CAT(a, b) DGW_CAT2(a, b)
namespace dgw {
int DGW_CAT(upload_ops_, REALNS)(const void* host_ops, size_t bytes, void* stream) {
  if (bytes != sizeof(AllOps<NORD, REAL>)) return int(cudaErrorInvalidValue);
  const int rc = REALNS::prepare_n<NORD>();
  if (rc) return rc;
  return int(cudaMemcpyToSymbolAsync(REALNS::c_ops, host_ops, bytes, 0, cudaMemcpyHostToDevice, cudaStream_t(stream)));
}
int DGW_CAT(launch_stage_, REALNS)(const StageArgs<REAL>& a, bool rk, void* stream, void* stream_t, void* ev_fork,
                                   void* ev_join) {
  return REALNS::launch_stage_n<NORD>(a, rk, cudaStream_t(stream), cudaStream_t(stream_t), cudaEvent_t(ev_fork),
                                      cudaEvent_t(ev_join));
}
int DGW_CAT(launch_pack_, REALNS)(const DevMesh<REAL>& m, const REAL* canon, REAL* packed, bool unpack, void* stream) {
  return REALNS::launch_pack_n<NORD>(m, canon, packed, unpack, cudaStream_t(stream));
}
int DGW_CAT(launch_energy_, REALNS)(const DevMesh<REAL>& m, const REAL* q, void* stream) {
  return REALNS::launch_energy_n<NORD>(m, q, cudaStream_t(stream));
}
int DGW_CAT(launch_sample_, REALNS)(const DevMesh<REAL>& m, const REAL* q, REAL* out, int nshots, void* stream) {
  const int n = nshots * m.nrec;
  if (n > 0) REALNS::k_sample<NORD><<<(n + 127) / 128, 128, 0, cudaStream_t(stream)>>>(m, q, out, nshots);
  return int(cudaGetLastError());
}
int DGW_CAT(launch_inject_, REALNS)(const DevMesh<REAL>& m, REAL* muq, REAL* x, const REAL* resid, int nshots, REAL b5,
                                    void* stream) {
  const int n = nshots * m.nrgrp;
  if (n > 0) REALNS::k_inject<NORD><<<(n + 127) / 128, 128, 0, cudaStream_t(stream)>>>(m, muq, x, resid, nshots, b5);
  return int(cudaGetLastError());
}
int DGW_CAT(launch_grad_, REALNS)(const DevMesh<REAL>& m, const REAL* x, const REAL* q, const REAL* r, double dt,
                                  int flux, int bc, double* gk, double* gr, double* gz, void* stream) {
  if (m.nblk_w > 0) {
    constexpr int bytes = REALNS::grad_smem_bytes<NORD>();
    if (bytes > 227 * 1024) return int(cudaErrorInvalidConfiguration);
    if (m.nblk_t > 0)
      REALNS::k_wedge_grad<NORD, true><<<m.nblk_w, 32 * (NORD + 1), bytes, cudaStream_t(stream)>>>(m, x, q, r, dt, flux,
                                                                                                  bc, gk, gr, gz);
    else
      REALNS::k_wedge_grad<NORD, false><<<m.nblk_w, 32 * (NORD + 1), bytes, cudaStream_t(stream)>>>(m, x, q, r, dt, flux,
                                                                                                   bc, gk, gr, gz);
  }
  return int(cudaGetLastError());
}
int DGW_CAT(launch_tgrad_, REALNS)(const DevMesh<REAL>& m, const REAL* x, const REAL* q, const REAL* r, double dt,
                                   int flux, int bc, double* gk, double* gr, void* stream) {
  if (m.nblk_t > 0) {
    constexpr int bytes = REALNS::tgrad_smem_bytes<NORD>();
    REALNS::k_tet_grad<NORD><<<m.nblk_t, 128, bytes, cudaStream_t(stream)>>>(m, x, q, r, dt, flux, bc, gk, gr);
  }
  return int(cudaGetLastError());
}
int DGW_CAT(launch_wait_expire_, REALNS)(int* err, void* stream) {
  REALNS::k_wait_expire<<<1, 32, 0, cudaStream_t(stream)>>>(err);
  return int(cudaGetLastError());
}
int DGW_CAT(launch_set_clock_, REALNS)(double* clock, double t, void* stream) {
  REALNS::k_set_clock<<<1, 32, 0, cudaStream_t(stream)>>>(clock, t);
  return int(cudaGetLastError());
}
int DGW_CAT(launch_clock_, REALNS)(double* clock, double dt, void* stream) {
  REALNS::k_clock<<<1, 32, 0, cudaStream_t(stream)>>>(clock, dt);
  return int(cudaGetLastError());
}
}  // namespace dgw
