// Internal types shared by the host library and the CUDA kernels.
//
// Device data layout (all element-indexed arrays are structure-of-arrays over
// 32-element blocks so that one warp reads one 128-byte line per item):
//   field buffers  wedge region [nblk_w][Np_w][32][4 fields], then
//                  tet region   [nblk_t][Np_t][32][4 fields]   (packed state,
//                  a node's four fields adjacent: one 16-byte access)
//   w_vid   [6][Kw_pad]  vertex ids            t_vid  [4][Kt_pad]
//   w_nbr   [5][Kw_pad]  neighbour index       t_nbr  [4][Kt_pad]
//   w_code  [5][Kw_pad]  orientation code      t_code [4][Kt_pad]
//   w_mat   [3][Kw_pad]  kappa, 1/rho, rho c   t_mat  [3][Kt_pad]
//   vx, vy, vz [nverts]
// Neighbour index -1 marks a boundary face.  Orientation codes:
//   triangle face: bit 6 set = neighbour is a tet; bits 4-5 = neighbour's face;
//                  bits 0-3 = triangle symmetry p0*3+p1 (see RefElems::tri_perm)
//   wedge quad face: (neighbour's triangle edge) * 2 + reversed
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace dgw {

constexpr int kB = 32;            // elements per block (one warp lane each)
constexpr int kMaxOrder = 5;
constexpr int kCodeTet = 64;
// energy partial sums held by the allocation-free entry point (128 elements each)
constexpr int kStaticPartials = 1 << 16;

__host__ __device__ constexpr int nt_of(int N) { return (N + 1) * (N + 2) / 2; }
__host__ __device__ constexpr int npw_of(int N) { return nt_of(N) * (N + 1); }
__host__ __device__ constexpr int npt_of(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
// Packed lower triangle of the wedge mass factor, Nt (Nt + 1) / 2 entries
// (entry (i, l <= i) at i (i + 1) / 2 + l), stored per 32-wedge block in
// groups of four: entry q of lane l at ((q / 4) * 32 + l) * 4 + q % 4, so a
// lane reads four consecutive entries with one 16-byte access.
__host__ __device__ constexpr int nl4_of(int N) { return (nt_of(N) * (nt_of(N) + 1) / 2 + 3) / 4; }

// Operator tables placed in device constant memory, one configuration at a time.
template <int N, typename real>
struct WedgeOps {
  static constexpr int Nt = nt_of(N), Nq = N + 1;
  real Dr[Nt * Nt], Ds[Nt * Nt], M[Nt * Nt], Ma[3][Nt * Nt];
  real Dt[Nq * Nq], ell0[Nq], ellN[Nq], Mea[Nq * Nq], Meb[Nq * Nq], M1[Nq * Nq], gll[Nq];
  // The same matrices by output pairs for packed multiply-adds: entry (h, l)
  // of XP is {X[2h][l], X[2h + 1][l]} at XP[(h * cols + l) * 2] (a zero row
  // completes an odd row count), so one 8-byte constant operand feeds two rows.
  static constexpr int Nh = (Nt + 1) / 2, Nqh = (Nq + 1) / 2;
  alignas(16) real MP[Nh * Nt * 2];
  alignas(16) real DrP[Nh * Nt * 2];
  alignas(16) real DsP[Nh * Nt * 2];
  alignas(16) real MeaP[Nqh * Nq * 2];
  alignas(16) real MebP[Nqh * Nq * 2];
  alignas(16) real MaP[3][Nh * Nt * 2];
};

template <int N>
struct Tables {
  static constexpr int Nt = nt_of(N), Nq = N + 1;
  int8_t tri_perm[9][Nt];
  int8_t edge[3][Nq];
  int8_t tet_face[4][Nt];
};

// (the tet operators live in global memory, in the tet stage's shared-memory
// image t_ops, so the constant bank holds wedge operators and tables only)
template <int N, typename real>
struct AllOps {
  WedgeOps<N, real> w;
  Tables<N> tab;
};

// Point source in the pressure equation: rhs_p += amp R(f0, t - t0) g, with
// g = kappa_k (M^k)^{-1} l(x_s) precomputed on the host (Np reals at goff).
// receiver: pressure sampled by l(x_r) (table rec_l); the adjoint injects
// (M^k)^{-1} l(x_r) (table rec_g, kappa applied in the kernel)
struct RecDev {
  int type;   // 6 wedge, 4 tet
  int elem;   // index within its element type (one shot)
  int loff;   // offset of l(x_r) and of (M^k)^{-1} l(x_r) in their tables
  int pad;
};
// receivers sharing one element, consecutive in the receiver list
struct RecGroup {
  int type, elem, r0, nr;
};

struct SourceDev {
  int type;   // 6 wedge, 4 tet
  int elem;   // index within its element type
  int goff;   // offset of g in the source vector table
  int pad;
  double f0, t0, amp;
};
constexpr int kMaxSources = 4096;  // device entries: (source, shot) pairs
constexpr int kMaxReceivers = 65536;

template <typename real>
struct DevMesh {
  int Kw = 0, Kw_pad = 0, nblk_w = 0;
  const int* w_vid = nullptr;
  const int* w_nbr = nullptr;
  const int* w_code = nullptr;
  const real* w_mat = nullptr;
  const int64_t* w_canon = nullptr;  // canonical node offset of each wedge
  int Kt = 0, Kt_pad = 0, nblk_t = 0;
  const int* t_vid = nullptr;
  const int* t_nbr = nullptr;
  const int* t_code = nullptr;
  const real* t_mat = nullptr;
  const int64_t* t_canon = nullptr;
  const real* vx = nullptr;
  const real* vy = nullptr;
  const real* vz = nullptr;
  int64_t tet_off = 0;               // first real of the tet region in a field buffer
  int64_t total_nodes = 0;           // canonical nodes
  int* err = nullptr;                // device error word
  double* partials = nullptr;        // per-block energy partial sums
  double* energy = nullptr;          // final energy
  const real* tet_mass = nullptr;    // reference tet mass matrix (energy only)
  const SourceDev* src = nullptr;    // point sources
  const real* src_g = nullptr;       // their vectors g
  int nsrc = 0;
  double* clock = nullptr;           // simulation time of the current step
  const real* w_fac = nullptr;       // stored mass factors per wedge block, or null (factor in the stage)
  const real* w_xyz = nullptr;       // per wedge block [12][32]: bottom x, y; bottom and top z
  const real* t_xyz = nullptr;       // per tet block [12][32]: x, y, z of the four vertices
  const real* t_ops = nullptr;       // tet stage operators, shared-memory image
  const RecDev* rec = nullptr;       // receivers (same for every shot)
  const RecGroup* rgrp = nullptr;    // receivers grouped by element
  const int* rperm = nullptr;        // receiver indices sorted by element (groups index this)
  const real* rec_l = nullptr;
  const real* rec_g = nullptr;
  int nrec = 0, nrgrp = 0;
  int Kw1 = 0, Kt1 = 0;              // wedges / tets of one shot
  int shot_group = 1, nshots = 1;    // virtual element of (shot s, element i): (s / G) K1 G + i G + s % G
  const int* w_srng = nullptr;       // per wedge block [begin, end) of its entries in src
  const int* t_srng = nullptr;       // per tet block likewise
};

template <typename real>
struct StageArgs {
  DevMesh<real> m;
  const real* q_in = nullptr;   // packed state read by this stage
  real* q_out = nullptr;        // RK: packed next state; RHS mode: packed rhs
  real* res = nullptr;          // RK residual (unused in RHS mode)
  real rk_a = 0, rk_b = 0, dt = 0;
  real rk_g = 1;                // RK: q_out = rk_g q_in + rk_b res' (1 in the forward method)
  real* rhs_out = nullptr;      // RK: also store the stage right-hand side here (optional)
  double c_stage = 0;           // stage time = *clock + c_stage * dt
  int bc = 1, flux = 0;
  int wedge_bpc = 0;            // wedge blocks per CTA: 0 = the default for the mass mode
  int op = 0;                   // kOpFFMA, or a tensor-core variant (FP32 fields)
  int split = 0;                // wedge stage split over field pairs: 1 yes, otherwise no
  int tri_far = 0;              // some wedge's triangle-face neighbour is a tet or in another block
};

enum : int { kErrTimeout = 1, kErrNonfinite = 2 };

// Virtual element of (shot s, type-local element i) with K1 elements of the
// type per shot and shots in groups of G: the G shots of a group are
// consecutive for each element (G = 1: shot-major, G = shots: shot-inner).
__host__ __device__ inline int64_t shot_vid(int64_t s, int64_t i, int64_t K1, int64_t G) {
  return (s / G) * (K1 * G) + i * G + s % G;
}

// How the wedge stage applies the shared triangle operators (M^tri, D_r,
// D_s): FP32 FMA chains on the CUDA cores, or warp-level tensor-core MMA with
// 3xTF32 (about FP32 accuracy), TF32 or BF16 operands and FP32 accumulation
// (FP32 fields only).
enum : int { kOpFFMA = 0, kOpTF32x3 = 1, kOpTF32 = 2, kOpBF16 = 3 };
// Per-warp operand tiles of the tensor-core applies: Nt rows of 128 columns
// (element lane * 4 + field), column c of row r stored at r * 128 +
// (c XOR ((r mod 4) * 8)): the lanes' 16-byte row accesses, the B-operand
// loads (4 rows x 8 columns) and the 64-bit C stores (half-warps over 4 rows)
// all hit distinct banks.
constexpr int kTP = 4 * 32;
__host__ __device__ constexpr int tile_at(int r, int c) { return r * kTP + (c ^ ((r & 3) << 3)); }

// Launchers, one set per (precision, order) translation unit k_<p>_n<N>.cu;
// all return 0 or a cudaError_t value.
#define DGW_DECLARE_LAUNCHERS(P, T, N)                                                              \
  int upload_ops_##P##n##N(const void* host_ops, size_t bytes, void* stream);                      \
  int launch_stage_##P##n##N(const StageArgs<T>& a, bool rk, void* stream, void* stream_t, void* ev_fork, \
                             void* ev_join);                                                       \
  int launch_pack_##P##n##N(const DevMesh<T>& m, const T* canon, T* packed, bool unpack, void* s); \
  int launch_energy_##P##n##N(const DevMesh<T>& m, const T* q, void* stream);                      \
  int launch_clock_##P##n##N(double* clock, double dt, void* stream);                              \
  int launch_wait_expire_##P##n##N(int* err, void* stream);                                        \
  int launch_set_clock_##P##n##N(double* clock, double t, void* stream);                           \
  int launch_sample_##P##n##N(const DevMesh<T>& m, const T* q, T* out, int nshots, void* stream);     \
  int launch_inject_##P##n##N(const DevMesh<T>& m, T* muq, T* x, const T* resid, int nshots, T b5,     \
                              void* stream);                                                       \
  int launch_grad_##P##n##N(const DevMesh<T>& m, const T* x, const T* q, const T* r, double dt, int flux, \
                            int bc, double* gk, double* gr, double* gz, void* stream);            \
  int launch_tgrad_##P##n##N(const DevMesh<T>& m, const T* x, const T* q, const T* r, double dt, int flux, \
                             int bc, double* gk, double* gr, void* stream);
DGW_DECLARE_LAUNCHERS(f32, float, 1)
DGW_DECLARE_LAUNCHERS(f32, float, 2)
DGW_DECLARE_LAUNCHERS(f32, float, 3)
DGW_DECLARE_LAUNCHERS(f32, float, 4)
DGW_DECLARE_LAUNCHERS(f32, float, 5)
DGW_DECLARE_LAUNCHERS(f64, double, 1)
DGW_DECLARE_LAUNCHERS(f64, double, 2)
DGW_DECLARE_LAUNCHERS(f64, double, 3)
DGW_DECLARE_LAUNCHERS(f64, double, 4)
DGW_DECLARE_LAUNCHERS(f64, double, 5)

// allocation-free energy (energy_static.cu)
int energy_static_scratch(int device, double** out);
template <typename real>
int launch_energy_static(int N, const DevMesh<real>& m, const real* q, const real* wops, double* scratch, int nblocks,
                         void* stream);

}  // namespace dgw
