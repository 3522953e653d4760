// C ABI of the DG library (see include/dgwedge.h).
//
// Host side: mesh validation (vertically mapped wedges, Section 3.2;
// positive Jacobians), face matching by vertex sets, face-node orientation
// codes, reference operators (refel.cpp), packing into the device blob, and
// the stage/step driver (LSRK45 stages replayed from a captured CUDA graph).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/dgwedge.h"
#include "dg_internal.hpp"
#include "refel.hpp"

using namespace dgw;

namespace {
// dispatch to the (precision, order) translation units
#define DGW_SWITCH_N(N, P, CALL)  \
  switch (N) {                    \
    case 1: return P##n1 CALL;    \
    case 2: return P##n2 CALL;    \
    case 3: return P##n3 CALL;    \
    case 4: return P##n4 CALL;    \
    case 5: return P##n5 CALL;    \
  }                               \
  return int(cudaErrorInvalidValue);

int upload_ops(int N, bool dbl, const void* p, size_t n, void* s) {
  if (dbl) {
    DGW_SWITCH_N(N, upload_ops_f64, (p, n, s))
  } else {
    DGW_SWITCH_N(N, upload_ops_f32, (p, n, s))
  }
}
int stage_f32(int N, const StageArgs<float>& a, bool rk, void* s, void* st, void* ef, void* ej) {
  DGW_SWITCH_N(N, launch_stage_f32, (a, rk, s, st, ef, ej))
}
int stage_f64(int N, const StageArgs<double>& a, bool rk, void* s, void* st, void* ef, void* ej) {
  DGW_SWITCH_N(N, launch_stage_f64, (a, rk, s, st, ef, ej))
}
int pack_f32(int N, const DevMesh<float>& m, const float* c, float* p, bool u, void* s) {
  DGW_SWITCH_N(N, launch_pack_f32, (m, c, p, u, s))
}
int pack_f64(int N, const DevMesh<double>& m, const double* c, double* p, bool u, void* s) {
  DGW_SWITCH_N(N, launch_pack_f64, (m, c, p, u, s))
}
int energy_f32(int N, const DevMesh<float>& m, const float* q, void* s) { DGW_SWITCH_N(N, launch_energy_f32, (m, q, s)) }
int clock_f32(int N, double* c, double dt, void* s) { DGW_SWITCH_N(N, launch_clock_f32, (c, dt, s)) }
int clock_f64(int N, double* c, double dt, void* s) { DGW_SWITCH_N(N, launch_clock_f64, (c, dt, s)) }
int set_clock_f32(int N, double* c, double t, void* s) { DGW_SWITCH_N(N, launch_set_clock_f32, (c, t, s)) }
int set_clock_f64(int N, double* c, double t, void* s) { DGW_SWITCH_N(N, launch_set_clock_f64, (c, t, s)) }
int wait_expire_f32(int N, int* e, void* s) { DGW_SWITCH_N(N, launch_wait_expire_f32, (e, s)) }
int wait_expire_f64(int N, int* e, void* s) { DGW_SWITCH_N(N, launch_wait_expire_f64, (e, s)) }
int energy_f64(int N, const DevMesh<double>& m, const double* q, void* s) { DGW_SWITCH_N(N, launch_energy_f64, (m, q, s)) }
int sample_f32(int N, const DevMesh<float>& m, const float* q, float* o, int ns, void* s) {
  DGW_SWITCH_N(N, launch_sample_f32, (m, q, o, ns, s))
}
int sample_f64(int N, const DevMesh<double>& m, const double* q, double* o, int ns, void* s) {
  DGW_SWITCH_N(N, launch_sample_f64, (m, q, o, ns, s))
}
int inject_f32(int N, const DevMesh<float>& m, float* mu, float* x, const float* r, int ns, float b5, void* s) {
  DGW_SWITCH_N(N, launch_inject_f32, (m, mu, x, r, ns, b5, s))
}
int inject_f64(int N, const DevMesh<double>& m, double* mu, double* x, const double* r, int ns, double b5, void* s) {
  DGW_SWITCH_N(N, launch_inject_f64, (m, mu, x, r, ns, b5, s))
}
int grad_f32(int N, const DevMesh<float>& m, const float* x, const float* q, const float* r, double dt, int fl, int bc,
             double* gk, double* gr, double* gz, void* s) {
  DGW_SWITCH_N(N, launch_grad_f32, (m, x, q, r, dt, fl, bc, gk, gr, gz, s))
}
int grad_f64(int N, const DevMesh<double>& m, const double* x, const double* q, const double* r, double dt, int fl, int bc,
             double* gk, double* gr, double* gz, void* s) {
  DGW_SWITCH_N(N, launch_grad_f64, (m, x, q, r, dt, fl, bc, gk, gr, gz, s))
}
int tgrad_f32(int N, const DevMesh<float>& m, const float* x, const float* q, const float* r, double dt, int fl, int bc,
              double* gk, double* gr, void* s) {
  DGW_SWITCH_N(N, launch_tgrad_f32, (m, x, q, r, dt, fl, bc, gk, gr, s))
}
int tgrad_f64(int N, const DevMesh<double>& m, const double* x, const double* q, const double* r, double dt, int fl,
              int bc, double* gk, double* gr, void* s) {
  DGW_SWITCH_N(N, launch_tgrad_f64, (m, x, q, r, dt, fl, bc, gk, gr, s))
}
}  // namespace

namespace {

const int kWedgeFaceVerts[5][4] = {{0, 1, 2, -1}, {3, 4, 5, -1}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}};
const int kTetFaceVerts[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

struct FaceKey {
  int64_t v[4];
  bool operator==(const FaceKey& o) const { return v[0] == o.v[0] && v[1] == o.v[1] && v[2] == o.v[2] && v[3] == o.v[3]; }
};
struct FaceKeyHash {
  size_t operator()(const FaceKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 4; ++i) {
      h ^= uint64_t(k.v[i]) + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
      h *= 1099511628211ull;
    }
    return size_t(h);
  }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// devices (bit mask) whose constant banks hold the operators of (order, precision)
uint64_t g_loaded[2 * (kMaxOrder + 1)] = {0};

}  // namespace

struct dg_ctx {
  mutable std::string err;
  // mesh (input order)
  int64_t nverts = 0, K = 0;
  std::vector<double> VX;
  std::vector<int64_t> EToV;
  std::vector<uint8_t> etype;
  // per element: type-local index and type-local lists
  std::vector<int64_t> local;  // index within its type
  std::vector<int64_t> wedges, tets;
  // connectivity (input order): neighbour element and its face per face (-1 boundary)
  std::vector<std::array<int64_t, 5>> nbr;
  std::vector<std::array<int, 5>> nface;
  std::vector<std::array<int, 5>> code;  // orientation code (see dg_internal.hpp)
  // order
  int N = 0;
  std::unique_ptr<RefElems> ref;
  std::vector<int64_t> node_off;  // canonical node offset per element
  int64_t wedge_nodes = 0, tet_nodes = 0;
  // material
  std::vector<double> c2, rho;
  // options
  int bc = DG_BC_RIGID, flux = DG_FLUX_UPWIND, prec = DG_F32;
  int mass = DG_MASS_STORED;
  int op = DG_OPS_FP32;  // how the wedge stage applies the shared triangle operators
  // shots: independent copies of the state on the same mesh, advanced together
  int64_t shots = 1;
  // shots per group G (dg_set_shot_group; 0 = all shots, DG_SHOTS_INNER): the G
  // shots of a group are neighbouring lanes for each element
  int64_t shot_group = 1;
  int64_t group() const { return shot_group == 0 ? shots : shot_group; }
  // launch variant chosen by dg_autotune: wedge blocks per CTA (0 = default) and
  // whether the stored mass factor is bypassed (factor recomputed in the stage)
  int tuned_bpc = 0;
  bool tuned_onthefly = false;
  int tuned_split = 0;  // wedge stage split over field pairs: 1 yes, -1 no, 0 the default for the order
  bool tri_far = false;  // some wedge's triangle-face neighbour is a tet or lies in another 32-block
  // adjoint workspace (caller-owned): mu_Q, two stage-input buffers, residual,
  // forward stage states Q_1..Q_4 and a scratch output, stage right-hand sides
  // r_1..r_5, then the kappa and rho gradients (doubles per device wedge)
  unsigned char* adj = nullptr;
  int adj_x = 0;
  // the gradient launches of the reverse sweep run on their own stream beside
  // the adjoint stage of the same Runge-Kutta stage (fork and join events)
  cudaStream_t grad_stream = nullptr;
  cudaEvent_t ev_gfork = nullptr, ev_gjoin = nullptr;
  // point sources (pressure equation)
  struct Source {
    int64_t elem;
    int64_t shot;  // -1: every shot
    double f0, t0, amp;
    std::vector<double> g;  // (M^k)^{-1} l(x_s), element node order (kappa applied in the kernels)
  };
  std::vector<Source> sources;
  // receivers: pressure sampled at points (adjoint misfits)
  struct Receiver {
    int64_t elem;
    std::vector<double> l, g;  // l(x_r) and (M^k)^{-1} l(x_r), element node order
  };
  std::vector<Receiver> receivers;
  // binding
  bool bound = false;
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  // meshes with both element types: the tet stage's stream, forked from and
  // joined back into the launching stream by these events
  cudaStream_t tet_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void* d_mesh = nullptr;
  void* d_q[2] = {nullptr, nullptr};
  void* d_res = nullptr;
  int cur = 0;
  double t = 0.0;
  DevMesh<float> m32;
  DevMesh<double> m64;
  size_t mesh_bytes = 0, field_bytes = 0;
  size_t wops_off = 0;  // offset of the wedge energy operators in the mesh blob
  std::vector<unsigned char> ops_host;
  // graphs: one LSRK step starting from buffer 0 / 1 for a given dt
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  double gdt[2] = {0.0, 0.0};

  int fail(int code_, const std::string& msg) const {
    err = msg;
    return code_;
  }
};

namespace {

int cuda_fail(dg_ctx* c, cudaError_t e, const char* what) {
  return c->fail(DG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Whether some device wedge's triangle-face neighbour is a tet or lies in
// another 32-wedge block (a column that straddles two blocks, the wedge/tet
// interface, shot-inner layouts): then the wedge stage requests those traces
// before its quadrilateral faces.  From the neighbour tables of a filled blob
// (w_nbr and w_code are [face][padded device wedge]).
bool triangle_neighbours_far(const std::vector<unsigned char>& blob, size_t off_nbr, size_t off_code, int64_t VKw) {
  const int64_t Kwp = (VKw + kB - 1) / kB * kB;
  const int* wn = reinterpret_cast<const int*>(blob.data() + off_nbr);
  const int* wc = reinterpret_cast<const int*>(blob.data() + off_code);
  for (int f = 0; f < 2; ++f)
    for (int64_t v = 0; v < VKw; ++v) {
      const int n = wn[f * Kwp + v];
      if (n >= 0 && ((wc[f * Kwp + v] & kCodeTet) != 0 || (n / kB) != (v / kB))) return true;
    }
  return false;
}

int64_t nblk(int64_t K) { return (K + kB - 1) / kB; }

// ----------------------------------------------------------------- operators
template <int NN, typename real>
void fill_ops(const RefElems& R, std::vector<unsigned char>& out) {
  AllOps<NN, real> o;
  std::memset(&o, 0, sizeof(o));
  const int Nt = R.Nt, Nq = R.Nq;
  for (int i = 0; i < Nt; ++i)
    for (int l = 0; l < Nt; ++l) {
      o.w.Dr[i * Nt + l] = real(R.Dr(i, l));
      o.w.Ds[i * Nt + l] = real(R.Ds(i, l));
      o.w.M[i * Nt + l] = real(R.Mt(i, l));
      for (int a = 0; a < 3; ++a) o.w.Ma[a][i * Nt + l] = real(R.Ma[a](i, l));
    }
  for (int m = 0; m < Nq; ++m) {
    for (int n = 0; n < Nq; ++n) {
      o.w.Dt[m * Nq + n] = real(R.D1(m, n));
      o.w.Mea[m * Nq + n] = real(R.Mea(m, n));
      o.w.Meb[m * Nq + n] = real(R.Meb(m, n));
      o.w.M1[m * Nq + n] = real(R.M1(m, n));
    }
    o.w.ell0[m] = real(R.ell0[m]);
    o.w.ellN[m] = real(R.ellN[m]);
    o.w.gll[m] = real(R.gll[m]);
  }
  // output-pair copies (rows 2h and 2h + 1; zero past the last row)
  auto pairs = [](const real* X, int rows, int cols, real* XP) {
    for (int h = 0; h < (rows + 1) / 2; ++h)
      for (int l = 0; l < cols; ++l)
        for (int b = 0; b < 2; ++b) XP[(h * cols + l) * 2 + b] = 2 * h + b < rows ? X[(2 * h + b) * cols + l] : real(0);
  };
  pairs(o.w.M, Nt, Nt, o.w.MP);
  pairs(o.w.Dr, Nt, Nt, o.w.DrP);
  pairs(o.w.Ds, Nt, Nt, o.w.DsP);
  pairs(o.w.Mea, Nq, Nq, o.w.MeaP);
  pairs(o.w.Meb, Nq, Nq, o.w.MebP);
  for (int a = 0; a < 3; ++a) pairs(o.w.Ma[a], Nt, Nt, o.w.MaP[a]);
  for (int c = 0; c < 9; ++c)
    for (int k = 0; k < Nt; ++k) o.tab.tri_perm[c][k] = R.tri_perm[c].empty() ? 0 : int8_t(R.tri_perm[c][k]);
  for (int e = 0; e < 3; ++e)
    for (int m = 0; m < Nq; ++m) o.tab.edge[e][m] = int8_t(R.edge_nodes[e][m]);
  for (int f = 0; f < 4; ++f)
    for (int k = 0; k < Nt; ++k) o.tab.tet_face[f][k] = int8_t(R.tet_face_nodes[f][k]);
  out.resize(sizeof(o));
  std::memcpy(out.data(), &o, sizeof(o));
}

void build_ops(dg_ctx* c) {
  const bool dbl = c->prec == DG_F64;
  const RefElems& R = *c->ref;
  switch (c->N) {
    case 1: dbl ? fill_ops<1, double>(R, c->ops_host) : fill_ops<1, float>(R, c->ops_host); break;
    case 2: dbl ? fill_ops<2, double>(R, c->ops_host) : fill_ops<2, float>(R, c->ops_host); break;
    case 3: dbl ? fill_ops<3, double>(R, c->ops_host) : fill_ops<3, float>(R, c->ops_host); break;
    case 4: dbl ? fill_ops<4, double>(R, c->ops_host) : fill_ops<4, float>(R, c->ops_host); break;
    case 5: dbl ? fill_ops<5, double>(R, c->ops_host) : fill_ops<5, float>(R, c->ops_host); break;
  }
}

// Operator tables depend only on (order, precision); each lives in the
// constant bank of its own translation unit, uploaded once per device.
int ensure_ops(dg_ctx* c) {
  const int key = c->N * 2 + (c->prec == DG_F64 ? 1 : 0);
  const uint64_t bit = uint64_t(1) << (c->device & 63);
  if (g_loaded[key] & bit) return DG_OK;
  const int rc = upload_ops(c->N, c->prec == DG_F64, c->ops_host.data(), c->ops_host.size(), c->stream);
  if (rc) return cuda_fail(c, cudaError_t(rc), "operator upload");
  const cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "operator upload synchronize");
  g_loaded[key] |= bit;
  return DG_OK;
}

// ----------------------------------------------------------------- geometry helpers
int nfaces_of(uint8_t t) { return t == DG_WEDGE ? 5 : 4; }

// vertex list (3 ids) of a triangle face in that element's face vertex order
void tri_face_vertices(const dg_ctx* c, int64_t k, int f, int64_t* out) {
  if (c->etype[k] == DG_WEDGE) {
    for (int i = 0; i < 3; ++i) out[i] = c->EToV[k * 6 + kWedgeFaceVerts[f][i]];
  } else {
    for (int i = 0; i < 3; ++i) out[i] = c->EToV[k * 6 + kTetFaceVerts[f][i]];
  }
}

double wedge_stable_ratio(const dg_ctx* c, int64_t k) {
  const double* V = c->VX.data();
  auto P = [&](int a, int d) { return V[c->EToV[k * 6 + a] * 3 + d]; };
  const double xr = 0.5 * (P(1, 0) - P(0, 0)), xs = 0.5 * (P(2, 0) - P(0, 0));
  const double yr = 0.5 * (P(1, 1) - P(0, 1)), ys = 0.5 * (P(2, 1) - P(0, 1));
  const double A = xr * ys - xs * yr;
  double h[3], hs = 0;
  for (int a = 0; a < 3; ++a) {
    h[a] = P(a + 3, 2) - P(a, 2);
    hs += h[a];
  }
  const double vol = (2.0 / 3.0) * A * hs;
  double amax = 0.0;
  for (int top = 0; top < 2; ++top) {
    const int o = top ? 3 : 0;
    double ab[3], ac[3];
    for (int d = 0; d < 3; ++d) {
      ab[d] = P(o + 1, d) - P(o, d);
      ac[d] = P(o + 2, d) - P(o, d);
    }
    const double cx = ab[1] * ac[2] - ab[2] * ac[1], cy = ab[2] * ac[0] - ab[0] * ac[2], cz = ab[0] * ac[1] - ab[1] * ac[0];
    amax = std::max(amax, 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz));
  }
  for (int e = 0; e < 3; ++e) {
    const int a = e, b = (e + 1) % 3;
    const double L = std::hypot(P(b, 0) - P(a, 0), P(b, 1) - P(a, 1));
    amax = std::max(amax, L * 0.5 * (h[a] + h[b]));
  }
  return amax / vol;
}

double tet_det(const dg_ctx* c, int64_t k) {
  const double* V = c->VX.data();
  double G[3][3];
  for (int m = 0; m < 3; ++m)
    for (int d = 0; d < 3; ++d) G[d][m] = V[c->EToV[k * 6 + m + 1] * 3 + d] - V[c->EToV[k * 6] * 3 + d];
  return G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) - G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
         G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
}

double tet_stable_ratio(const dg_ctx* c, int64_t k) {
  const double* V = c->VX.data();
  const double vol = tet_det(c, k) / 6.0;
  double amax = 0.0;
  for (int f = 0; f < 4; ++f) {
    const int64_t a = c->EToV[k * 6 + kTetFaceVerts[f][0]], b = c->EToV[k * 6 + kTetFaceVerts[f][1]],
                  d = c->EToV[k * 6 + kTetFaceVerts[f][2]];
    double ab[3], ad[3];
    for (int i = 0; i < 3; ++i) {
      ab[i] = V[b * 3 + i] - V[a * 3 + i];
      ad[i] = V[d * 3 + i] - V[a * 3 + i];
    }
    const double cx = ab[1] * ad[2] - ab[2] * ad[1], cy = ab[2] * ad[0] - ab[0] * ad[2], cz = ab[0] * ad[1] - ab[1] * ad[0];
    amax = std::max(amax, 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz));
  }
  return amax / vol;
}

// ----------------------------------------------------------------- blob
struct BlobLayout {
  size_t w_vid, w_nbr, w_code, w_mat, w_canon, t_vid, t_nbr, t_code, t_mat, t_canon, vx, vy, vz, err, partials, energy,
      tmass, wops, src, srcg, clock, wfac, wxyz, txyz, tops, wsrng, tsrng, rec, rgrp, rperm, recl, recg, total;
};

// Shots are laid out shot-major over the type-local element lists: the
// device-side (virtual) element s K + i is type-local element i of shot s.
int64_t vKw(const dg_ctx* c) { return c->shots * int64_t(c->wedges.size()); }
int64_t vKt(const dg_ctx* c) { return c->shots * int64_t(c->tets.size()); }
int64_t nsrc_dev(const dg_ctx* c) {
  int64_t n = 0;
  for (const auto& sc : c->sources) n += sc.shot < 0 ? c->shots : 1;
  return n;
}

BlobLayout blob_layout(const dg_ctx* c) {
  const size_t rs = c->prec == DG_F64 ? 8 : 4;
  const int64_t Kwp = nblk(vKw(c)) * kB, Ktp = nblk(vKt(c)) * kB;
  const int64_t nparts = (nblk(vKw(c)) + 3) / 4 + (nblk(vKt(c)) + 3) / 4 + 1;
  BlobLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.w_vid = take(6 * Kwp * 4);
  L.w_nbr = take(5 * Kwp * 4);
  L.w_code = take(5 * Kwp * 4);
  L.w_mat = take(3 * Kwp * rs);
  L.w_canon = take(Kwp * 8);
  L.t_vid = take(4 * Ktp * 4);
  L.t_nbr = take(4 * Ktp * 4);
  L.t_code = take(4 * Ktp * 4);
  L.t_mat = take(3 * Ktp * rs);
  L.t_canon = take(Ktp * 8);
  L.vx = take(c->nverts * rs);
  L.vy = take(c->nverts * rs);
  L.vz = take(c->nverts * rs);
  L.err = take(16);
  L.partials = take(nparts * 8);
  L.energy = take(8);
  L.tmass = take(size_t(npt_of(c->N)) * npt_of(c->N) * rs);
  L.wops = take(size_t(3 * nt_of(c->N) * nt_of(c->N) + (c->N + 1) * (c->N + 1)) * rs);
  L.src = take(sizeof(SourceDev) * size_t(std::max<int64_t>(1, nsrc_dev(c))));
  // per block [begin, end) of its sources in the element-sorted source list
  L.wsrng = take(size_t(2) * nblk(vKw(c)) * 4 + 4);
  L.tsrng = take(size_t(2) * nblk(vKt(c)) * 4 + 4);
  {
    const size_t nr = std::max<size_t>(1, c->receivers.size());
    size_t nl = 1;
    for (const auto& r : c->receivers) nl += r.l.size();
    L.rec = take(sizeof(RecDev) * nr);
    L.rgrp = take(sizeof(RecGroup) * nr);
    L.rperm = take(sizeof(int) * nr);
    L.recl = take(nl * rs);
    L.recg = take(nl * rs);
  }
  size_t ng = 0;
  for (const auto& sc : c->sources) ng += sc.g.size();
  L.srcg = take((ng > 0 ? ng : 1) * rs);
  L.clock = take(sizeof(double));
  // stored mass factors: per wedge block [NL4][32][4], the stage's shared-memory layout
  const int64_t nl4 = nl4_of(c->N);
  L.wfac = take(c->mass == DG_MASS_STORED ? size_t(Kwp * nl4 * 4) * rs : 0);
  // per wedge block [12][32]: x, y of the three bottom vertices, z of the six
  L.wxyz = take(size_t(Kwp) * 12 * rs);
  // per tet block [12][32]: x, y, z of the four vertices
  L.txyz = take(size_t(Ktp) * 12 * rs);
  // tet stage operators in the stage's shared-memory image: [l][i] (D_r, D_s, D_t, 0)(i, l),
  // then the lift per warp chunk of C = ceil(Np/4) output nodes, [warp][f Nt + k][c < CP]
  {
    const int np = npt_of(c->N), ch = (np + 3) / 4, cp = (ch + 3) / 4 * 4;
    L.tops = take(size_t(4 * np * np + 4 * 4 * nt_of(c->N) * cp) * rs);
  }
  L.total = o;
  return L;
}

template <typename real>
void fill_blob(const dg_ctx* c, const BlobLayout& L, std::vector<unsigned char>& blob) {
  blob.assign(L.total, 0);
  const int64_t Kw = int64_t(c->wedges.size()), Kt = int64_t(c->tets.size());
  const int64_t S = c->shots, T = c->wedge_nodes + c->tet_nodes;
  const int64_t VKw = S * Kw, VKt = S * Kt;
  const int64_t Kwp = nblk(VKw) * kB, Ktp = nblk(VKt) * kB;
  // virtual id of (shot s, input element n): shots in groups of G, a group's
  // shots consecutive per element (G = 1 shot-major, G = S shot-inner)
  const int64_t G = c->group();
  auto vid = [&](int64_t s, int64_t n) { return shot_vid(s, c->local[n], c->etype[n] == DG_WEDGE ? Kw : Kt, G); };
  // (shot, type-local element) of a virtual element
  auto vsplit = [&](int64_t v, int64_t K1, int64_t& sh, int64_t& el) {
    const int64_t r = v % (K1 * G);
    el = r / G;
    sh = (v / (K1 * G)) * G + r % G;
  };
  int* w_vid = reinterpret_cast<int*>(blob.data() + L.w_vid);
  int* w_nbr = reinterpret_cast<int*>(blob.data() + L.w_nbr);
  int* w_code = reinterpret_cast<int*>(blob.data() + L.w_code);
  real* w_mat = reinterpret_cast<real*>(blob.data() + L.w_mat);
  int64_t* w_canon = reinterpret_cast<int64_t*>(blob.data() + L.w_canon);
  for (int64_t w = 0; w < Kwp; ++w) {
    const bool real_slot = w < VKw;  // padding replicates a valid element with no neighbours
    int64_t s = 0, el = 0;
    if (real_slot) vsplit(w, Kw, s, el);
    const int64_t k = c->wedges[el];
    for (int v = 0; v < 6; ++v) w_vid[v * Kwp + w] = int(c->EToV[k * 6 + v]);
    for (int f = 0; f < 5; ++f) {
      const int64_t n = real_slot ? c->nbr[k][f] : -1;
      w_nbr[f * Kwp + w] = (n < 0) ? -1 : int(vid(s, n));
      w_code[f * Kwp + w] = (n < 0) ? 0 : c->code[k][f];
    }
    {
      real* xyz = reinterpret_cast<real*>(blob.data() + L.wxyz) + (w / kB) * 12 * kB + (w % kB);
      const int64_t* ev = &c->EToV[k * 6];
      for (int a = 0; a < 3; ++a) {
        xyz[(0 + a) * kB] = real(c->VX[ev[a] * 3 + 0]);
        xyz[(3 + a) * kB] = real(c->VX[ev[a] * 3 + 1]);
        xyz[(6 + a) * kB] = real(c->VX[ev[a] * 3 + 2]);
        xyz[(9 + a) * kB] = real(c->VX[ev[a + 3] * 3 + 2]);
      }
    }
    const double cc = std::sqrt(c->c2[k]);
    w_mat[0 * Kwp + w] = real(c->rho[k] * c->c2[k]);
    w_mat[1 * Kwp + w] = real(1.0 / c->rho[k]);
    w_mat[2 * Kwp + w] = real(c->rho[k] * cc);
    if (real_slot) w_canon[w] = 4 * s * T + c->node_off[k];
  }
  int* t_vid = reinterpret_cast<int*>(blob.data() + L.t_vid);
  int* t_nbr = reinterpret_cast<int*>(blob.data() + L.t_nbr);
  int* t_code = reinterpret_cast<int*>(blob.data() + L.t_code);
  real* t_mat = reinterpret_cast<real*>(blob.data() + L.t_mat);
  int64_t* t_canon = reinterpret_cast<int64_t*>(blob.data() + L.t_canon);
  for (int64_t t = 0; t < Ktp; ++t) {
    const bool real_slot = t < VKt;
    int64_t s = 0, el = 0;
    if (real_slot) vsplit(t, Kt, s, el);
    const int64_t k = c->tets[el];
    for (int v = 0; v < 4; ++v) t_vid[v * Ktp + t] = int(c->EToV[k * 6 + v]);
    for (int f = 0; f < 4; ++f) {
      const int64_t n = real_slot ? c->nbr[k][f] : -1;
      t_nbr[f * Ktp + t] = (n < 0) ? -1 : int(vid(s, n));
      t_code[f * Ktp + t] = (n < 0) ? 0 : c->code[k][f];
    }
    {
      real* xyz = reinterpret_cast<real*>(blob.data() + L.txyz) + (t / kB) * 12 * kB + (t % kB);
      for (int v = 0; v < 4; ++v)
        for (int d = 0; d < 3; ++d) xyz[(v * 3 + d) * kB] = real(c->VX[c->EToV[k * 6 + v] * 3 + d]);
    }
    const double cc = std::sqrt(c->c2[k]);
    t_mat[0 * Ktp + t] = real(c->rho[k] * c->c2[k]);
    t_mat[1 * Ktp + t] = real(1.0 / c->rho[k]);
    t_mat[2 * Ktp + t] = real(c->rho[k] * cc);
    if (real_slot) t_canon[t] = 4 * s * T + c->node_off[k];
  }
  // sources: one device entry per (source, shot), sorted by (type, virtual element);
  // each element block records the range of its entries
  {
    struct Ent {
      int type;
      int64_t elem;
      size_t src;
    };
    std::vector<Ent> ents;
    for (size_t i = 0; i < c->sources.size(); ++i) {
      const auto& sc = c->sources[i];
      for (int64_t sh = 0; sh < S; ++sh)
        if (sc.shot < 0 || sc.shot == sh) ents.push_back({int(c->etype[sc.elem]), vid(sh, sc.elem), i});
    }
    std::stable_sort(ents.begin(), ents.end(),
                     [](const Ent& x, const Ent& y) { return x.type != y.type ? x.type < y.type : x.elem < y.elem; });
    std::vector<int> goffs(c->sources.size());
    real* sg = reinterpret_cast<real*>(blob.data() + L.srcg);
    int goff = 0;
    for (size_t i = 0; i < c->sources.size(); ++i) {
      goffs[i] = goff;
      for (size_t n = 0; n < c->sources[i].g.size(); ++n) sg[goff + n] = real(c->sources[i].g[n]);
      goff += int(c->sources[i].g.size());
    }
    SourceDev* sd = reinterpret_cast<SourceDev*>(blob.data() + L.src);
    int* wr = reinterpret_cast<int*>(blob.data() + L.wsrng);
    int* tr = reinterpret_cast<int*>(blob.data() + L.tsrng);
    for (size_t i = 0; i < ents.size(); ++i) {
      const auto& sc = c->sources[ents[i].src];
      sd[i].type = ents[i].type;
      sd[i].elem = int(ents[i].elem);
      sd[i].goff = goffs[ents[i].src];
      sd[i].pad = 0;
      sd[i].f0 = sc.f0;
      sd[i].t0 = sc.t0;
      sd[i].amp = sc.amp;
      int* rng = (ents[i].type == DG_WEDGE ? wr : tr) + 2 * (ents[i].elem / kB);
      if (rng[1] == rng[0]) rng[0] = int(i);  // first entry of the block (ranges start empty)
      rng[1] = int(i) + 1;
    }
  }
  {
    // receivers in the caller's order; groups of receivers sharing an element
    // (sorted by element) for the deterministic adjoint load
    RecDev* rd = reinterpret_cast<RecDev*>(blob.data() + L.rec);
    real* rl = reinterpret_cast<real*>(blob.data() + L.recl);
    real* rg = reinterpret_cast<real*>(blob.data() + L.recg);
    int off = 0;
    const size_t nr = c->receivers.size();
    for (size_t r = 0; r < nr; ++r) {
      const auto& rc = c->receivers[r];
      rd[r].type = c->etype[rc.elem];
      rd[r].elem = int(c->local[rc.elem]);
      rd[r].loff = off;
      rd[r].pad = 0;
      for (size_t n = 0; n < rc.l.size(); ++n) {
        rl[off + n] = real(rc.l[n]);
        rg[off + n] = real(rc.g[n]);
      }
      off += int(rc.l.size());
    }
    std::vector<int> perm(nr);
    for (size_t r = 0; r < nr; ++r) perm[r] = int(r);
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
      return rd[a].type != rd[b].type ? rd[a].type < rd[b].type : rd[a].elem < rd[b].elem;
    });
    int* rp = reinterpret_cast<int*>(blob.data() + L.rperm);
    RecGroup* gp = reinterpret_cast<RecGroup*>(blob.data() + L.rgrp);
    int ng = 0;
    for (size_t i = 0; i < nr; ++i) {
      rp[i] = perm[i];
      if (i == 0 || rd[perm[i]].type != rd[perm[i - 1]].type || rd[perm[i]].elem != rd[perm[i - 1]].elem)
        gp[ng++] = RecGroup{rd[perm[i]].type, rd[perm[i]].elem, int(i), 0};
      gp[ng - 1].nr++;
    }
  }
  real* vx = reinterpret_cast<real*>(blob.data() + L.vx);
  real* vy = reinterpret_cast<real*>(blob.data() + L.vy);
  real* vz = reinterpret_cast<real*>(blob.data() + L.vz);
  real* tm = reinterpret_cast<real*>(blob.data() + L.tmass);
  for (int i = 0; i < c->ref->Npt * c->ref->Npt; ++i) tm[i] = real(c->ref->tM.a[i]);
  // wedge energy operators: barycentric-weighted triangle masses, then the line mass
  {
    const RefElems& R = *c->ref;
    const int np = R.Npt, nt = R.Nt, ch = (np + 3) / 4, cp = (ch + 3) / 4 * 4;
    real* to = reinterpret_cast<real*>(blob.data() + L.tops);
    for (int l = 0; l < np; ++l)
      for (int i = 0; i < np; ++i) {
        real* v = to + (size_t(l) * np + i) * 4;
        v[0] = real(R.tDr(i, l));
        v[1] = real(R.tDs(i, l));
        v[2] = real(R.tDt(i, l));
        v[3] = real(0);
      }
    real* lt = to + size_t(4) * np * np;
    for (int w = 0; w < 4; ++w)
      for (int fk = 0; fk < 4 * nt; ++fk)
        for (int cc = 0; cc < cp; ++cc) {
          const int i = w * ch + cc;
          lt[(size_t(w) * 4 * nt + fk) * cp + cc] = (cc < ch && i < np) ? real(R.tLIFT(i, fk)) : real(0);
        }
  }
  real* wo = reinterpret_cast<real*>(blob.data() + L.wops);
  const int nt2 = c->ref->Nt * c->ref->Nt;
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < nt2; ++i) wo[a * nt2 + i] = real(c->ref->Ma[a].a[i]);
  for (int i = 0; i < c->ref->Nq * c->ref->Nq; ++i) wo[3 * nt2 + i] = real(c->ref->M1.a[i]);
  for (int64_t v = 0; v < c->nverts; ++v) {
    vx[v] = real(c->VX[v * 3 + 0]);
    vy[v] = real(c->VX[v * 3 + 1]);
    vz[v] = real(c->VX[v * 3 + 2]);
  }
  if (c->mass == DG_MASS_STORED) {
    // M^{tri,k} = sum_a J_a M_a with J_a = A h_a / 2 at the three columns
    // (Lemma 3.1, bi-unit reference: A = x_r y_s - x_s y_r), factored L L^T in
    // double; entry (i, l <= i) at i (i + 1) / 2 + l with 1 / L_ii on the diagonal
    const RefElems& R = *c->ref;
    const int nt = R.Nt, nl = nt * (nt + 1) / 2;
    real* fac = reinterpret_cast<real*>(blob.data() + L.wfac);
    std::vector<double> Mk(size_t(nt) * nt), Lk(size_t(nt) * nt);
    std::vector<real> one(size_t(Kw) * nl);  // per type-local wedge, then copied to every shot's slot
    for (int64_t w = 0; w < Kw; ++w) {
      const int64_t k = c->wedges[w];
      const int64_t* ev = &c->EToV[k * 6];
      const double* P[6];
      for (int v = 0; v < 6; ++v) P[v] = &c->VX[ev[v] * 3];
      const double A = 0.25 * ((P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]));
      double J[3];
      for (int a = 0; a < 3; ++a) J[a] = 0.5 * A * (P[a + 3][2] - P[a][2]);
      for (int i = 0; i < nt * nt; ++i) Mk[i] = J[0] * R.Ma[0].a[i] + J[1] * R.Ma[1].a[i] + J[2] * R.Ma[2].a[i];
      for (int i = 0; i < nt; ++i) {
        for (int l = 0; l <= i; ++l) {
          double sum = Mk[size_t(i) * nt + l];
          for (int q = 0; q < l; ++q) sum -= Lk[size_t(i) * nt + q] * Lk[size_t(l) * nt + q];
          Lk[size_t(i) * nt + l] = (l < i) ? sum / Lk[size_t(l) * nt + l] : std::sqrt(sum);
        }
      }
      for (int i = 0; i < nt; ++i)
        for (int l = 0; l <= i; ++l)
          one[size_t(w) * nl + i * (i + 1) / 2 + l] = real(l < i ? Lk[size_t(i) * nt + l] : 1.0 / Lk[size_t(i) * nt + i]);
    }
    const int64_t nl4 = nl4_of(c->N);
    for (int64_t w = 0; w < Kwp; ++w) {
      int64_t sh = 0, lw = 0;
      if (w < VKw) vsplit(w, Kw, sh, lw);
      const int64_t b = w / kB, lane = w % kB;
      for (int q = 0; q < nl4 * 4; ++q)
        fac[((b * nl4 + q / 4) * kB + lane) * 4 + q % 4] = q < nl ? one[size_t(lw) * nl + q] : real(0);
    }
  }
}

template <typename real>
void fill_devmesh(const dg_ctx* c, const BlobLayout& L, DevMesh<real>& m) {
  unsigned char* b = static_cast<unsigned char*>(c->d_mesh);
  const int64_t Kw = vKw(c), Kt = vKt(c);
  m.Kw = int(Kw);
  m.Kw_pad = int(nblk(Kw) * kB);
  m.nblk_w = int(nblk(Kw));
  m.Kt = int(Kt);
  m.Kt_pad = int(nblk(Kt) * kB);
  m.nblk_t = int(nblk(Kt));
  m.w_vid = reinterpret_cast<const int*>(b + L.w_vid);
  m.w_nbr = reinterpret_cast<const int*>(b + L.w_nbr);
  m.w_code = reinterpret_cast<const int*>(b + L.w_code);
  m.w_mat = reinterpret_cast<const real*>(b + L.w_mat);
  m.w_canon = reinterpret_cast<const int64_t*>(b + L.w_canon);
  m.t_vid = reinterpret_cast<const int*>(b + L.t_vid);
  m.t_nbr = reinterpret_cast<const int*>(b + L.t_nbr);
  m.t_code = reinterpret_cast<const int*>(b + L.t_code);
  m.t_mat = reinterpret_cast<const real*>(b + L.t_mat);
  m.t_canon = reinterpret_cast<const int64_t*>(b + L.t_canon);
  m.vx = reinterpret_cast<const real*>(b + L.vx);
  m.vy = reinterpret_cast<const real*>(b + L.vy);
  m.vz = reinterpret_cast<const real*>(b + L.vz);
  m.err = reinterpret_cast<int*>(b + L.err);
  m.partials = reinterpret_cast<double*>(b + L.partials);
  m.energy = reinterpret_cast<double*>(b + L.energy);
  m.tet_mass = reinterpret_cast<const real*>(b + L.tmass);
  m.src = reinterpret_cast<const SourceDev*>(b + L.src);
  m.src_g = reinterpret_cast<const real*>(b + L.srcg);
  m.nsrc = int(nsrc_dev(c));
  m.w_srng = reinterpret_cast<const int*>(b + L.wsrng);
  m.rec = reinterpret_cast<const RecDev*>(b + L.rec);
  m.rgrp = reinterpret_cast<const RecGroup*>(b + L.rgrp);
  m.rperm = reinterpret_cast<const int*>(b + L.rperm);
  m.rec_l = reinterpret_cast<const real*>(b + L.recl);
  m.rec_g = reinterpret_cast<const real*>(b + L.recg);
  m.nrec = int(c->receivers.size());
  {
    int ng = 0;
    std::vector<std::pair<int, int64_t>> keys;
    for (const auto& r : c->receivers) keys.push_back({int(c->etype[r.elem]), c->local[r.elem]});
    std::sort(keys.begin(), keys.end());
    ng = int(std::unique(keys.begin(), keys.end()) - keys.begin());
    m.nrgrp = ng;
  }
  m.Kw1 = int(c->wedges.size());
  m.Kt1 = int(c->tets.size());
  m.shot_group = int(c->group());
  m.nshots = int(c->shots);
  m.t_srng = reinterpret_cast<const int*>(b + L.tsrng);
  m.clock = reinterpret_cast<double*>(b + L.clock);
  m.w_fac = c->mass == DG_MASS_STORED ? reinterpret_cast<const real*>(b + L.wfac) : nullptr;
  m.w_xyz = reinterpret_cast<const real*>(b + L.wxyz);
  m.t_xyz = reinterpret_cast<const real*>(b + L.txyz);
  m.t_ops = reinterpret_cast<const real*>(b + L.tops);
  m.tet_off = int64_t(m.nblk_w) * 4 * npw_of(c->N) * kB;
  m.total_nodes = c->wedge_nodes + c->tet_nodes;
}

size_t field_bytes_of(const dg_ctx* c) {
  const size_t rs = c->prec == DG_F64 ? 8 : 4;
  const int64_t nw = nblk(vKw(c)), nt = nblk(vKt(c));
  return align256(size_t(nw * 4 * npw_of(c->N) * kB + nt * 4 * npt_of(c->N) * kB) * rs);
}

// extra stage settings: the update coefficient on the input state, a store of the
// stage right-hand side, and whether the point sources are left out
struct StageExtra {
  double g = 1.0;
  void* rhs_out = nullptr;
  bool no_sources = false;
};

int launch_stage(dg_ctx* c, const void* q_in, void* q_out, void* res, double a, double b, double dt, bool rk,
                 cudaStream_t s, double cst = 0.0, const StageExtra& x = StageExtra()) {
  int rc;
  if (c->prec == DG_F64) {
    StageArgs<double> A;
    A.m = c->m64;
    A.q_in = static_cast<const double*>(q_in);
    A.q_out = static_cast<double*>(q_out);
    A.res = static_cast<double*>(res);
    A.rk_a = a;
    A.rk_b = b;
    A.dt = dt;
    A.c_stage = cst;
    A.bc = c->bc;
    A.flux = c->flux;
    A.wedge_bpc = c->tuned_bpc;
    if (c->tuned_onthefly) A.m.w_fac = nullptr;
    A.rk_g = x.g;
    A.rhs_out = static_cast<double*>(x.rhs_out);
    if (x.no_sources) A.m.nsrc = 0;
    rc = stage_f64(c->N, A, rk, s, c->tet_stream, c->ev_fork, c->ev_join);
  } else {
    StageArgs<float> A;
    A.m = c->m32;
    A.q_in = static_cast<const float*>(q_in);
    A.q_out = static_cast<float*>(q_out);
    A.res = static_cast<float*>(res);
    A.rk_a = float(a);
    A.rk_b = float(b);
    A.dt = float(dt);
    A.c_stage = cst;
    A.bc = c->bc;
    A.flux = c->flux;
    A.wedge_bpc = c->tuned_bpc;
    if (c->tuned_onthefly) A.m.w_fac = nullptr;
    A.op = c->op;
    A.split = c->tuned_split;
    A.tri_far = c->tri_far ? 1 : 0;
    A.rk_g = float(x.g);
    A.rhs_out = static_cast<float*>(x.rhs_out);
    if (x.no_sources) A.m.nsrc = 0;
    rc = stage_f32(c->N, A, rk, s, c->tet_stream, c->ev_fork, c->ev_join);
  }
  if (rc) return cuda_fail(c, cudaError_t(rc), "stage launch");
  return DG_OK;
}

int launch_pack(dg_ctx* c, const void* canon, void* packed, bool unpack, cudaStream_t s) {
  int rc;
  if (c->prec == DG_F64)
    rc = pack_f64(c->N, c->m64, static_cast<const double*>(canon), static_cast<double*>(packed), unpack, s);
  else
    rc = pack_f32(c->N, c->m32, static_cast<const float*>(canon), static_cast<float*>(packed), unpack, s);
  if (rc) return cuda_fail(c, cudaError_t(rc), "pack launch");
  return DG_OK;
}

int check_device_error(dg_ctx* c) {
  int h = 0;
  int* derr = (c->prec == DG_F64) ? c->m64.err : c->m32.err;
  cudaError_t e = cudaMemcpyAsync(&h, derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "device error check");
  if (h) {
    cudaMemsetAsync(derr, 0, sizeof(int), c->stream);
    cudaStreamSynchronize(c->stream);
    if (h & kErrTimeout) return c->fail(DG_ERR_TIMEOUT, "a bounded device-side wait ran out");
    if (h & kErrNonfinite) return c->fail(DG_ERR_NONFINITE, "non-finite value in the state");
  }
  return DG_OK;
}

// Makes the bound context's device current for the duration of an entry
// point and restores the caller's device afterwards, so work, symbol lookups
// and stream operations always address the device whose memory was bound.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(const dg_ctx* c) {
    if (!c->bound) return;
    int cur = -1;
    err = cudaGetDevice(&cur);
    if (err == cudaSuccess && cur != c->device) {
      err = cudaSetDevice(c->device);
      if (err == cudaSuccess) prev = cur;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

void drop_graphs(dg_ctx* c) {
  for (int i = 0; i < 2; ++i) {
    if (c->gexec[i]) cudaGraphExecDestroy(c->gexec[i]);
    c->gexec[i] = nullptr;
  }
}

}  // namespace

// =========================================================================== ABI
extern "C" {

int dg_mesh_create(dg_ctx** out, int64_t nverts, const double* VX, int64_t nelem, const int64_t* EToV,
                   const uint8_t* etype) {
  if (!out || !VX || !EToV || !etype || nverts <= 0 || nelem <= 0) return DG_ERR_ARG;
  *out = nullptr;
  std::unique_ptr<dg_ctx> c(new dg_ctx);
  c->nverts = nverts;
  c->K = nelem;
  c->VX.assign(VX, VX + nverts * 3);
  c->EToV.assign(EToV, EToV + nelem * 6);
  c->etype.assign(etype, etype + nelem);
  c->local.assign(nelem, -1);
  c->nbr.assign(nelem, {-1, -1, -1, -1, -1});
  c->nface.assign(nelem, {-1, -1, -1, -1, -1});
  c->code.assign(nelem, {0, 0, 0, 0, 0});
  for (int64_t k = 0; k < nelem; ++k) {
    const uint8_t t = etype[k];
    if (t != DG_WEDGE && t != DG_TET) {
      *out = c.release();
      return (*out)->fail(DG_ERR_ARG, "element " + std::to_string(k) + ": unknown element type");
    }
    const int nv = (t == DG_WEDGE) ? 6 : 4;
    for (int v = 0; v < nv; ++v) {
      const int64_t id = EToV[k * 6 + v];
      if (id < 0 || id >= nverts) {
        *out = c.release();
        return (*out)->fail(DG_ERR_MESH, "element " + std::to_string(k) + ": vertex id out of range");
      }
    }
    if (t == DG_WEDGE) {
      c->local[k] = int64_t(c->wedges.size());
      c->wedges.push_back(k);
    } else {
      c->local[k] = int64_t(c->tets.size());
      c->tets.push_back(k);
    }
  }
  if (c->wedges.size() >= (1u << 30) || c->tets.size() >= (1u << 30)) {
    *out = c.release();
    return (*out)->fail(DG_ERR_ARG, "too many elements");
  }
  // validation: vertically mapped wedges with positive Jacobian, positive tets
  for (int64_t k = 0; k < nelem; ++k) {
    const double* V = c->VX.data();
    if (etype[k] == DG_WEDGE) {
      auto P = [&](int a, int d) { return V[EToV[k * 6 + a] * 3 + d]; };
      double scale = 0.0;
      for (int a = 0; a < 6; ++a)
        for (int d = 0; d < 3; ++d) scale = std::max(scale, std::fabs(P(a, d) - P(0, d)));
      for (int a = 0; a < 3; ++a)
        if (std::fabs(P(a, 0) - P(a + 3, 0)) > 1e-10 * scale || std::fabs(P(a, 1) - P(a + 3, 1)) > 1e-10 * scale) {
          *out = c.release();
          return (*out)->fail(DG_ERR_MESH, "wedge " + std::to_string(k) + " is not vertically mapped");
        }
      const double A = (P(1, 0) - P(0, 0)) * (P(2, 1) - P(0, 1)) - (P(2, 0) - P(0, 0)) * (P(1, 1) - P(0, 1));
      bool ok = A > 0;
      for (int a = 0; a < 3; ++a) ok = ok && (P(a + 3, 2) - P(a, 2) > 0);
      if (!ok) {
        *out = c.release();
        return (*out)->fail(DG_ERR_MESH, "wedge " + std::to_string(k) +
                                             " has J <= 0 (bottom must be counter-clockwise seen from +z, top above bottom)");
      }
    } else {
      if (!(tet_det(c.get(), k) > 0)) {
        *out = c.release();
        return (*out)->fail(DG_ERR_MESH, "tet " + std::to_string(k) + " has J <= 0");
      }
    }
  }
  // face matching by vertex sets
  std::unordered_map<FaceKey, std::pair<int64_t, int>, FaceKeyHash> open;
  open.reserve(size_t(nelem) * 3);
  for (int64_t k = 0; k < nelem; ++k) {
    const bool w = etype[k] == DG_WEDGE;
    for (int f = 0; f < nfaces_of(etype[k]); ++f) {
      FaceKey key{{-1, -1, -1, -1}};
      int nv = 3;
      if (w) {
        nv = (f < 2) ? 3 : 4;
        for (int i = 0; i < nv; ++i) key.v[i] = EToV[k * 6 + kWedgeFaceVerts[f][i]];
      } else {
        for (int i = 0; i < 3; ++i) key.v[i] = EToV[k * 6 + kTetFaceVerts[f][i]];
      }
      std::sort(key.v, key.v + nv);
      auto it = open.find(key);
      if (it == open.end()) {
        open.emplace(key, std::make_pair(k, f));
      } else {
        // matched faces stay in the table (marked by f2 < 0) so that a third
        // element on the same face is detected
        const int64_t k2 = it->second.first;
        const int f2 = it->second.second;
        if (f2 < 0) {
          *out = c.release();
          return (*out)->fail(DG_ERR_MESH, "a face of element " + std::to_string(k) + " is shared by more than two elements");
        }
        c->nbr[k][f] = k2;
        c->nface[k][f] = f2;
        c->nbr[k2][f2] = k;
        c->nface[k2][f2] = f;
        it->second.second = -1;
      }
    }
  }
  // orientation codes
  for (int64_t k = 0; k < nelem; ++k) {
    for (int f = 0; f < nfaces_of(etype[k]); ++f) {
      const int64_t k2 = c->nbr[k][f];
      if (k2 < 0) continue;
      const int f2 = c->nface[k][f];
      const bool quad = etype[k] == DG_WEDGE && f >= 2;
      if (quad) {
        const int64_t a = EToV[k * 6 + kWedgeFaceVerts[f][0]], b = EToV[k * 6 + kWedgeFaceVerts[f][1]];
        const int64_t a2 = EToV[k2 * 6 + kWedgeFaceVerts[f2][0]], b2 = EToV[k2 * 6 + kWedgeFaceVerts[f2][1]];
        int rev;
        if (a == a2 && b == b2)
          rev = 0;
        else if (a == b2 && b == a2)
          rev = 1;
        else {
          *out = c.release();
          return (*out)->fail(DG_ERR_MESH, "wedges " + std::to_string(k) + " and " + std::to_string(k2) +
                                                " meet on a quad face with opposite vertical orientation");
        }
        c->code[k][f] = (f2 - 2) * 2 + rev;
      } else {
        int64_t own[3], oth[3];
        tri_face_vertices(c.get(), k, f, own);
        tri_face_vertices(c.get(), k2, f2, oth);
        int pos[3];
        for (int m = 0; m < 3; ++m) {
          pos[m] = -1;
          for (int i = 0; i < 3; ++i)
            if (oth[m] == own[i]) pos[m] = i;
        }
        c->code[k][f] = (etype[k2] == DG_TET ? kCodeTet : 0) | (f2 << 4) | (pos[0] * 3 + pos[1]);
      }
    }
  }
  c->c2.assign(nelem, 1.0);
  c->rho.assign(nelem, 1.0);
  *out = c.release();
  return DG_OK;
}

int dg_set_order(dg_ctx* c, int N) {
  if (!c) return DG_ERR_ARG;
  if (c->bound) return c->fail(DG_ERR_STATE, "dg_set_order after dg_bind");
  if (N < 1 || N > kMaxOrder) return c->fail(DG_ERR_ORDER, "order must be in 1..5");
  try {
    c->ref.reset(new RefElems(build_reference(N)));
  } catch (const std::exception& ex) {
    return c->fail(DG_ERR_ORDER, ex.what());
  }
  c->N = N;
  c->sources.clear();
  c->node_off.assign(c->K + 1, 0);
  c->wedge_nodes = c->tet_nodes = 0;
  for (int64_t k = 0; k < c->K; ++k) {
    const int np = c->etype[k] == DG_WEDGE ? c->ref->Npw : c->ref->Npt;
    c->node_off[k + 1] = c->node_off[k] + np;
    (c->etype[k] == DG_WEDGE ? c->wedge_nodes : c->tet_nodes) += np;
  }
  return DG_OK;
}

int dg_set_material(dg_ctx* c, const double* c2, const double* rho) {
  if (!c) return DG_ERR_ARG;
  if (!c2 || !rho) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (c->bound) return c->fail(DG_ERR_STATE, "dg_set_material after dg_bind");
  for (int64_t k = 0; k < c->K; ++k)
    if (!(c2[k] > 0) || !(rho[k] > 0) || !std::isfinite(c2[k]) || !std::isfinite(rho[k]))
      return c->fail(DG_ERR_ARG, "material of element " + std::to_string(k) + " must be positive and finite");
  c->c2.assign(c2, c2 + c->K);
  c->rho.assign(rho, rho + c->K);
  return DG_OK;
}

// The element holding (x, y, z) (lowest id on ties), the Lagrange basis values
// lv = l(x) of its nodes and g = (M^k)^{-1} l(x) (element node order); false
// when the point lies outside the mesh.
static bool point_vectors(const dg_ctx* c, double x, double y, double z, int64_t& elem, std::vector<double>& lv,
                          std::vector<double>& g) {
  const RefElems& R = *c->ref;
  const double* V = c->VX.data();
  const double tol = 1e-12;
  for (int64_t k = 0; k < c->K; ++k) {
    auto P = [&](int a, int d) { return V[c->EToV[k * 6 + a] * 3 + d]; };
    double ref[3];
    bool inside = false;
    if (c->etype[k] == DG_WEDGE) {
      // barycentric coordinates in the (affine) footprint, then t along the column
      const double a11 = P(1, 0) - P(0, 0), a12 = P(2, 0) - P(0, 0), a21 = P(1, 1) - P(0, 1), a22 = P(2, 1) - P(0, 1);
      const double det = a11 * a22 - a12 * a21;
      const double bx = x - P(0, 0), by = y - P(0, 1);
      const double l1 = (a22 * bx - a12 * by) / det, l2 = (a11 * by - a21 * bx) / det, l0 = 1.0 - l1 - l2;
      const double zb = l0 * P(0, 2) + l1 * P(1, 2) + l2 * P(2, 2), zt = l0 * P(3, 2) + l1 * P(4, 2) + l2 * P(5, 2);
      const double t = (2.0 * z - zb - zt) / (zt - zb);
      inside = l0 >= -tol && l1 >= -tol && l2 >= -tol && std::fabs(t) <= 1.0 + tol;
      ref[0] = 2.0 * l1 - 1.0;
      ref[1] = 2.0 * l2 - 1.0;
      ref[2] = t;
    } else {
      double G[3][3], Gi[3][3];
      for (int d = 0; d < 3; ++d)
        for (int m = 0; m < 3; ++m) G[d][m] = P(m + 1, d) - P(0, d);
      const double det = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) - G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
                         G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
      Gi[0][0] = (G[1][1] * G[2][2] - G[1][2] * G[2][1]) / det;
      Gi[0][1] = (G[0][2] * G[2][1] - G[0][1] * G[2][2]) / det;
      Gi[0][2] = (G[0][1] * G[1][2] - G[0][2] * G[1][1]) / det;
      Gi[1][0] = (G[1][2] * G[2][0] - G[1][0] * G[2][2]) / det;
      Gi[1][1] = (G[0][0] * G[2][2] - G[0][2] * G[2][0]) / det;
      Gi[1][2] = (G[0][2] * G[1][0] - G[0][0] * G[1][2]) / det;
      Gi[2][0] = (G[1][0] * G[2][1] - G[1][1] * G[2][0]) / det;
      Gi[2][1] = (G[0][1] * G[2][0] - G[0][0] * G[2][1]) / det;
      Gi[2][2] = (G[0][0] * G[1][1] - G[0][1] * G[1][0]) / det;
      const double b[3] = {x - P(0, 0), y - P(0, 1), z - P(0, 2)};
      double l[3];
      for (int m = 0; m < 3; ++m) l[m] = Gi[m][0] * b[0] + Gi[m][1] * b[1] + Gi[m][2] * b[2];
      inside = l[0] >= -tol && l[1] >= -tol && l[2] >= -tol && (1.0 - l[0] - l[1] - l[2]) >= -tol;
      for (int m = 0; m < 3; ++m) ref[m] = 2.0 * l[m] - 1.0;
    }
    if (!inside) continue;
    elem = k;
    if (c->etype[k] == DG_WEDGE) {
      // (M^k)^{-1} = (M^{tri,k})^{-1} (x) (M^1D)^{-1},  M^{tri,k} = sum_a J_a M_a
      const double A = 0.25 * ((P(1, 0) - P(0, 0)) * (P(2, 1) - P(0, 1)) - (P(2, 0) - P(0, 0)) * (P(1, 1) - P(0, 1)));
      Mat Mt(R.Nt, R.Nt), Mti, M1i;
      for (int a = 0; a < 3; ++a) {
        const double Ja = 0.5 * A * (P(a + 3, 2) - P(a, 2));
        for (size_t i = 0; i < Mt.a.size(); ++i) Mt.a[i] += Ja * R.Ma[a].a[i];
      }
      invert(Mt, Mti);
      invert(R.M1, M1i);
      std::vector<double> lt(R.Nt), l1(R.Nq), gt(R.Nt, 0.0), g1(R.Nq, 0.0);
      tri_lagrange(R, ref[0], ref[1], lt.data());
      line_lagrange(R, ref[2], l1.data());
      for (int i = 0; i < R.Nt; ++i)
        for (int l = 0; l < R.Nt; ++l) gt[i] += Mti(i, l) * lt[l];
      for (int j = 0; j < R.Nq; ++j)
        for (int l = 0; l < R.Nq; ++l) g1[j] += M1i(j, l) * l1[l];
      g.resize(R.Npw);
      lv.resize(R.Npw);
      for (int j = 0; j < R.Nq; ++j)
        for (int i = 0; i < R.Nt; ++i) {
          g[j * R.Nt + i] = gt[i] * g1[j];
          lv[j * R.Nt + i] = lt[i] * l1[j];
        }
    } else {
      const double J = tet_det(c, k) / 8.0;
      Mat Mi;
      invert(R.tM, Mi);
      lv.assign(R.Npt, 0.0);
      tet_lagrange(R, ref[0], ref[1], ref[2], lv.data());
      g.assign(R.Npt, 0.0);
      for (int i = 0; i < R.Npt; ++i) {
        for (int l = 0; l < R.Npt; ++l) g[i] += Mi(i, l) * lv[l];
        g[i] /= J;
      }
    }
    return true;
  }
  return false;
}


static int add_source(dg_ctx* c, int64_t shot, double x, double y, double z, double f0, double t0, double amp) {
  if (c->bound) return c->fail(DG_ERR_STATE, "dg_add_source after dg_bind");
  if (!c->N) return c->fail(DG_ERR_STATE, "dg_add_source needs dg_set_order first");
  if (!(f0 > 0) || !std::isfinite(t0) || !std::isfinite(amp))
    return c->fail(DG_ERR_ARG, "source frequency must be positive and t0, amp finite");
  if (shot >= c->shots) return c->fail(DG_ERR_ARG, "shot index out of range");
  if (nsrc_dev(c) + (shot < 0 ? c->shots : 1) > kMaxSources) return c->fail(DG_ERR_ARG, "too many sources");
  dg_ctx::Source sc;
  std::vector<double> lv;
  if (!point_vectors(c, x, y, z, sc.elem, lv, sc.g)) return c->fail(DG_ERR_ARG, "source point lies outside the mesh");
  sc.shot = shot;
  sc.f0 = f0;
  sc.t0 = t0;
  sc.amp = amp;
  c->sources.push_back(sc);
  return DG_OK;
}

int dg_add_receiver(dg_ctx* c, double x, double y, double z) {
  if (!c) return DG_ERR_ARG;
  if (c->bound) return c->fail(DG_ERR_STATE, "dg_add_receiver after dg_bind");
  if (!c->N) return c->fail(DG_ERR_STATE, "dg_add_receiver needs dg_set_order first");
  if (c->receivers.size() >= size_t(kMaxReceivers)) return c->fail(DG_ERR_ARG, "too many receivers");
  dg_ctx::Receiver rc;
  if (!point_vectors(c, x, y, z, rc.elem, rc.l, rc.g)) return c->fail(DG_ERR_ARG, "receiver point lies outside the mesh");
  c->receivers.push_back(rc);
  return int(c->receivers.size()) - 1;
}

int dg_add_source(dg_ctx* c, double x, double y, double z, double f0, double t0, double amp) {
  if (!c) return DG_ERR_ARG;
  return add_source(c, -1, x, y, z, f0, t0, amp);
}

int dg_add_shot_source(dg_ctx* c, int64_t shot, double x, double y, double z, double f0, double t0, double amp) {
  if (!c) return DG_ERR_ARG;
  if (shot < 0) return c->fail(DG_ERR_ARG, "shot index out of range");
  return add_source(c, shot, x, y, z, f0, t0, amp);
}

int dg_set_shots(dg_ctx* c, int64_t shots) {
  if (!c) return DG_ERR_ARG;
  if (c->bound) return c->fail(DG_ERR_STATE, "dg_set_shots after dg_bind");
  if (!c->N) return c->fail(DG_ERR_STATE, "dg_set_shots needs dg_set_order first");
  if (shots < 1) return c->fail(DG_ERR_ARG, "shots must be at least 1");
  for (const auto& sc : c->sources)
    if (sc.shot >= shots) return c->fail(DG_ERR_ARG, "a source refers to a shot beyond the new count");
  const int64_t K = int64_t(std::max(c->wedges.size(), c->tets.size()));
  if (shots * K >= (int64_t(1) << 30)) return c->fail(DG_ERR_ARG, "shots x elements exceeds 2^30");
  if (c->shot_group > 1 && shots % c->shot_group != 0)
    return c->fail(DG_ERR_ARG, "the shot group must divide the number of shots");
  c->shots = shots;
  return DG_OK;
}

int dg_set_shot_order(dg_ctx* c, int order) {
  if (!c) return DG_ERR_ARG;
  if (c->bound) return c->fail(DG_ERR_STATE, "dg_set_shot_order after dg_bind");
  if (order != DG_SHOTS_OUTER && order != DG_SHOTS_INNER) return c->fail(DG_ERR_ARG, "unknown shot order");
  c->shot_group = order == DG_SHOTS_INNER ? 0 : 1;
  return DG_OK;
}

int dg_set_shot_group(dg_ctx* c, int64_t group) {
  if (!c) return DG_ERR_ARG;
  if (c->bound) return c->fail(DG_ERR_STATE, "dg_set_shot_group after dg_bind");
  if (group < 1 || c->shots % group != 0) return c->fail(DG_ERR_ARG, "the shot group must divide the number of shots");
  c->shot_group = group;
  return DG_OK;
}

int dg_set_options(dg_ctx* c, int bc, int flux, int precision) {
  if (!c) return DG_ERR_ARG;
  if (c->bound) return c->fail(DG_ERR_STATE, "dg_set_options after dg_bind");
  if ((bc != DG_BC_DIRICHLET && bc != DG_BC_RIGID) || (flux != DG_FLUX_UPWIND && flux != DG_FLUX_CENTRAL) ||
      (precision != DG_F32 && precision != DG_F64))
    return c->fail(DG_ERR_ARG, "option out of range");
  if (precision != DG_F32 && c->op != DG_OPS_FP32)
    return c->fail(DG_ERR_ARG, "tensor-core operator applies need DG_F32 fields");
  c->bc = bc;
  c->flux = flux;
  c->prec = precision;
  return DG_OK;
}

int dg_set_mass_mode(dg_ctx* c, int mode) {
  if (!c) return DG_ERR_ARG;
  if (c->bound) return c->fail(DG_ERR_STATE, "dg_set_mass_mode after dg_bind");
  if (mode != DG_MASS_ONTHEFLY && mode != DG_MASS_STORED) return c->fail(DG_ERR_ARG, "mass mode out of range");
  c->mass = mode;
  return DG_OK;
}

int dg_set_op_precision(dg_ctx* c, int mode) {
  if (!c) return DG_ERR_ARG;
  if (c->bound) return c->fail(DG_ERR_STATE, "dg_set_op_precision after dg_bind");
  if (mode < DG_OPS_FP32 || mode > DG_OPS_BF16) return c->fail(DG_ERR_ARG, "operator precision out of range");
  if (mode != DG_OPS_FP32 && c->prec != DG_F32)
    return c->fail(DG_ERR_ARG, "tensor-core operator applies need DG_F32 fields");
  c->op = mode;
  return DG_OK;
}

int dg_num_nodes(const dg_ctx* c, int64_t* wn, int64_t* tn) {
  if (!c) return DG_ERR_ARG;
  if (!wn || !tn) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->N) return c->fail(DG_ERR_STATE, "call needs dg_set_order first");
  *wn = c->wedge_nodes;
  *tn = c->tet_nodes;
  return DG_OK;
}

int dg_node_coords(const dg_ctx* c, double* xyz) {
  if (!c) return DG_ERR_ARG;
  if (!xyz) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->N) return c->fail(DG_ERR_STATE, "call needs dg_set_order first");
  const RefElems& R = *c->ref;
  const int64_t tot = c->wedge_nodes + c->tet_nodes;
  const double* V = c->VX.data();
  for (int64_t k = 0; k < c->K; ++k) {
    const int64_t o = c->node_off[k];
    if (c->etype[k] == DG_WEDGE) {
      for (int j = 0; j < R.Nq; ++j)
        for (int i = 0; i < R.Nt; ++i) {
          const double r = R.tri_r[i], s = R.tri_s[i], t = R.gll[j];
          const double lam[3] = {-0.5 * (r + s), 0.5 * (1 + r), 0.5 * (1 + s)};
          const double lo = 0.5 * (1 - t), hi = 0.5 * (1 + t);
          for (int d = 0; d < 3; ++d) {
            double x = 0.0;
            for (int a = 0; a < 3; ++a)
              x += lam[a] * (lo * V[c->EToV[k * 6 + a] * 3 + d] + hi * V[c->EToV[k * 6 + a + 3] * 3 + d]);
            xyz[d * tot + o + j * R.Nt + i] = x;
          }
        }
    } else {
      for (int n = 0; n < R.Npt; ++n) {
        const double r = R.tet_r[n], s = R.tet_s[n], t = R.tet_t[n];
        const double lam[4] = {-0.5 * (1 + r + s + t), 0.5 * (1 + r), 0.5 * (1 + s), 0.5 * (1 + t)};
        for (int d = 0; d < 3; ++d) {
          double x = 0.0;
          for (int v = 0; v < 4; ++v) x += lam[v] * V[c->EToV[k * 6 + v] * 3 + d];
          xyz[d * tot + o + n] = x;
        }
      }
    }
  }
  return DG_OK;
}

int dg_face_neighbors(const dg_ctx* c, int64_t* out, int64_t* count) {
  if (!c) return DG_ERR_ARG;
  if (!count) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->N) return c->fail(DG_ERR_STATE, "call needs dg_set_order first");
  const RefElems& R = *c->ref;
  int64_t n = 0;
  for (int64_t k = 0; k < c->K; ++k) {
    const bool w = c->etype[k] == DG_WEDGE;
    for (int f = 0; f < nfaces_of(c->etype[k]); ++f) {
      const std::vector<int>& own = w ? R.wedge_face_nodes[f] : R.tet_face_nodes[f];
      const int64_t k2 = c->nbr[k][f];
      for (size_t q = 0; q < own.size(); ++q, ++n) {
        if (!out) continue;
        if (k2 < 0) {
          out[n] = -1;
          continue;
        }
        const int code = c->code[k][f];
        int node;
        if (w && f >= 2) {
          const int jj = int(q) / R.Nq, m = int(q) % R.Nq;
          const int ep = code >> 1, rev = code & 1;
          node = jj * R.Nt + R.edge_nodes[ep][rev ? R.N - m : m];
        } else {
          const int nf = (code >> 4) & 3, perm = code & 15;
          const int nk = R.tri_perm[perm][q];
          node = (c->etype[k2] == DG_TET) ? R.tet_face_nodes[nf][nk] : (nf ? R.N * R.Nt : 0) + nk;
        }
        out[n] = c->node_off[k2] + node;
      }
    }
  }
  *count = n;
  return DG_OK;
}

int dg_reference_operator(const dg_ctx* c, const char* name, double* out, int64_t* rows, int64_t* cols) {
  if (!c) return DG_ERR_ARG;
  if (!name || !rows || !cols) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->N) return c->fail(DG_ERR_STATE, "call needs dg_set_order first");
  const RefElems& R = *c->ref;
  const Mat* M = nullptr;
  const std::vector<double>* v = nullptr;
  const std::string s(name);
  if (s == "tri.Dr") M = &R.Dr;
  else if (s == "tri.Ds") M = &R.Ds;
  else if (s == "tri.M") M = &R.Mt;
  else if (s == "tri.M0") M = &R.Ma[0];
  else if (s == "tri.M1") M = &R.Ma[1];
  else if (s == "tri.M2") M = &R.Ma[2];
  else if (s == "line.D") M = &R.D1;
  else if (s == "line.M") M = &R.M1;
  else if (s == "line.Ma") M = &R.Mea;
  else if (s == "line.Mb") M = &R.Meb;
  else if (s == "tet.Dr") M = &R.tDr;
  else if (s == "tet.Ds") M = &R.tDs;
  else if (s == "tet.Dt") M = &R.tDt;
  else if (s == "tet.M") M = &R.tM;
  else if (s == "tet.LIFT") M = &R.tLIFT;
  else if (s == "tri.r") v = &R.tri_r;
  else if (s == "tri.s") v = &R.tri_s;
  else if (s == "line.r") v = &R.gll;
  else if (s == "line.ell0") v = &R.ell0;
  else if (s == "line.ellN") v = &R.ellN;
  else if (s == "tet.r") v = &R.tet_r;
  else if (s == "tet.s") v = &R.tet_s;
  else if (s == "tet.t") v = &R.tet_t;
  else return DG_ERR_ARG;
  if (M) {
    *rows = M->r;
    *cols = M->c;
    if (out) std::copy(M->a.begin(), M->a.end(), out);
  } else {
    *rows = int64_t(v->size());
    *cols = 1;
    if (out) std::copy(v->begin(), v->end(), out);
  }
  return DG_OK;
}

int dg_device_bytes(const dg_ctx* c, size_t* mesh_bytes, size_t* field_bytes) {
  if (!c) return DG_ERR_ARG;
  if (!mesh_bytes || !field_bytes) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->N) return c->fail(DG_ERR_STATE, "call needs dg_set_order first");
  *mesh_bytes = blob_layout(c).total;
  *field_bytes = field_bytes_of(c);
  return DG_OK;
}

int dg_bind(dg_ctx* c, void* d_mesh, void* d_q0, void* d_q1, void* d_res, void* stream) {
  if (!c) return DG_ERR_ARG;
  if (!d_mesh || !d_q0 || !d_q1 || !d_res) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->N) return c->fail(DG_ERR_STATE, "dg_bind before dg_set_order");
  if (c->bound) return c->fail(DG_ERR_STATE, "context already bound");
  if (c->shots % c->group() != 0) return c->fail(DG_ERR_ARG, "the shot group must divide the number of shots");
  if (c->op != DG_OPS_FP32 && nt_of(c->N) > 16)
    return c->fail(DG_ERR_ORDER, "tensor-core operator applies need N <= 4 (a slice in one 16-row tile)");
  for (void* p : {d_mesh, d_q0, d_q1, d_res})
    if (reinterpret_cast<uintptr_t>(p) % 256) return c->fail(DG_ERR_ARG, "device buffers must be 256-byte aligned");
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
  c->stream = static_cast<cudaStream_t>(stream);
  c->d_mesh = d_mesh;
  c->d_q[0] = d_q0;
  c->d_q[1] = d_q1;
  c->d_res = d_res;
  const BlobLayout L = blob_layout(c);
  std::vector<unsigned char> blob;
  if (c->prec == DG_F64) {
    fill_blob<double>(c, L, blob);
    fill_devmesh<double>(c, L, c->m64);
  } else {
    fill_blob<float>(c, L, blob);
    fill_devmesh<float>(c, L, c->m32);
  }
  c->mesh_bytes = L.total;
  c->wops_off = L.wops;
  c->field_bytes = field_bytes_of(c);
  c->tri_far = triangle_neighbours_far(blob, L.w_nbr, L.w_code, vKw(c));
  e = cudaMemcpyAsync(d_mesh, blob.data(), blob.size(), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "mesh upload");
  for (void* p : {d_q0, d_q1, d_res}) {
    e = cudaMemsetAsync(p, 0, c->field_bytes, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "state clear");
  }
  e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "bind synchronize");
  build_ops(c);
  const int rc = ensure_ops(c);
  if (rc) return rc;
  e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(c, e, "capture stream");
  if (vKw(c) > 0 && vKt(c) > 0) {
    e = cudaStreamCreateWithFlags(&c->tet_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(c, e, "tet stream");
  }
  c->bound = true;
  c->cur = 0;
  c->t = 0.0;
  return DG_OK;
}

namespace {
// The device address of a pinned, device-mapped host buffer, or nullptr for
// pageable memory.  With such a buffer the pack kernel reads or writes the
// host memory itself (over the CPU-GPU link) instead of a bulk copy plus a
// device-side pass.
const void* mapped_host_alias(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (at.type == cudaMemoryTypeHost && at.devicePointer != nullptr) ? at.devicePointer : nullptr;
}
}  // namespace

int dg_set_fields(dg_ctx* c, const void* q, int on_device) {
  if (!c) return DG_ERR_ARG;
  if (!q) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_set_fields before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc) return rc;
  const size_t rs = c->prec == DG_F64 ? 8 : 4;
  const size_t bytes = size_t(4) * c->shots * (c->wedge_nodes + c->tet_nodes) * rs;
  const void* src = q;
  if (!on_device) {
    src = mapped_host_alias(q);
    if (!src) {
      // pageable memory: pack reads a scratch copy into the current buffer
      cudaError_t e = cudaMemcpyAsync(c->d_q[1 - c->cur], q, bytes, cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "state upload");
      src = c->d_q[1 - c->cur];
    }
  }
  rc = launch_pack(c, src, c->d_q[c->cur], false, c->stream);
  if (rc) return rc;
  cudaError_t e = cudaMemsetAsync(c->d_res, 0, c->field_bytes, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "residual clear");
  e = cudaMemsetAsync((c->prec == DG_F64) ? c->m64.clock : c->m32.clock, 0, sizeof(double), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "clock reset");
  if (!on_device) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "state upload synchronize");
  }
  c->t = 0.0;
  return DG_OK;
}

int dg_get_fields(dg_ctx* c, void* q, int on_device) {
  if (!c) return DG_ERR_ARG;
  if (!q) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_get_fields before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);  // also opts the pack kernel in to its shared memory
  if (rc) return rc;
  const size_t rs = c->prec == DG_F64 ? 8 : 4;
  const size_t bytes = size_t(4) * c->shots * (c->wedge_nodes + c->tet_nodes) * rs;
  void* mapped = on_device ? nullptr : const_cast<void*>(mapped_host_alias(q));
  void* dst = on_device ? q : (mapped ? mapped : c->d_q[1 - c->cur]);
  rc = launch_pack(c, dst, c->d_q[c->cur], true, c->stream);
  if (rc) return rc;
  if (!on_device) {
    cudaError_t e = mapped ? cudaSuccess : cudaMemcpyAsync(q, dst, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "state download");
  }
  return DG_OK;
}

int dg_rhs(dg_ctx* c, const void* d_q, void* d_rhs) {
  if (!c) return DG_ERR_ARG;
  if (!d_q || !d_rhs) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_rhs before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc) return rc;
  void* A = c->d_q[1 - c->cur];
  void* B = c->d_res;
  rc = launch_pack(c, d_q, A, false, c->stream);
  if (rc) return rc;
  rc = launch_stage(c, A, B, nullptr, 0.0, 0.0, 0.0, false, c->stream);
  if (rc) return rc;
  rc = launch_pack(c, d_rhs, B, true, c->stream);
  if (rc) return rc;
  // the residual buffer was used as scratch; the next step starts from zero
  cudaError_t e = cudaMemsetAsync(c->d_res, 0, c->field_bytes, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "residual clear");
  return DG_OK;
}

int dg_step(dg_ctx* c, double dt, int64_t nsteps) {
  if (!c) return DG_ERR_ARG;
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_step before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  if (!(dt > 0) || nsteps < 0) return c->fail(DG_ERR_ARG, "dt must be positive and nsteps >= 0");
  int rc = ensure_ops(c);
  if (rc) return rc;
  for (int64_t n = 0; n < nsteps; ++n) {
    const int p = c->cur;
    if (!c->gexec[p] || c->gdt[p] != dt) {
      if (c->gexec[p]) {
        cudaGraphExecDestroy(c->gexec[p]);
        c->gexec[p] = nullptr;
      }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_fail(c, e, "graph capture begin");
      int src = p;
      int lrc = DG_OK;
      for (int s = 0; s < 5 && lrc == DG_OK; ++s) {
        lrc = launch_stage(c, c->d_q[src], c->d_q[1 - src], c->d_res, kLSRK_A[s], kLSRK_B[s], dt, true, c->cap_stream,
                           kLSRK_C[s]);
        src = 1 - src;
      }
      if (lrc == DG_OK) {
        double* clk = (c->prec == DG_F64) ? c->m64.clock : c->m32.clock;
        const int crc = (c->prec == DG_F64) ? clock_f64(c->N, clk, dt, c->cap_stream) : clock_f32(c->N, clk, dt, c->cap_stream);
        if (crc) lrc = cuda_fail(c, cudaError_t(crc), "clock launch");
      }
      e = cudaStreamEndCapture(c->cap_stream, &g);
      if (lrc) {
        if (g) cudaGraphDestroy(g);
        return lrc;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "graph capture end");
      e = cudaGraphInstantiate(&c->gexec[p], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
      c->gdt[p] = dt;
    }
    cudaError_t e = cudaGraphLaunch(c->gexec[p], c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    c->cur = 1 - c->cur;  // five stages: odd number of buffer swaps
    c->t += dt;
  }
  return DG_OK;
}

int dg_stage_times(dg_ctx* c, int nrep, double* us_w, double* us_t) {
  if (!c) return DG_ERR_ARG;
  if (nrep < 1 || !us_w || !us_t) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_stage_times before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc) return rc;
  *us_w = *us_t = 0.0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  if (e != cudaSuccess) {
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    return cuda_fail(c, e, "event create");
  }
  const DevMesh<float> m32 = c->m32;
  const DevMesh<double> m64 = c->m64;
  // element blocks of each type in the context's precision (only that mesh is filled)
  const int nbw = c->prec == DG_F64 ? m64.nblk_w : m32.nblk_w, nbt = c->prec == DG_F64 ? m64.nblk_t : m32.nblk_t;
  for (int type = 0; type < 2 && rc == DG_OK; ++type) {
    // restrict the stage to one element type (the other's blocks are not launched)
    if (type == 0) {
      c->m32.nblk_t = c->m64.nblk_t = 0;
      if (nbw == 0) continue;
    } else {
      c->m32 = m32;
      c->m64 = m64;
      c->m32.nblk_w = c->m64.nblk_w = 0;
      if (nbt == 0) continue;
    }
    e = cudaEventRecord(ev[0], c->stream);
    for (int r = 0; r < nrep && rc == DG_OK && e == cudaSuccess; ++r)
      rc = launch_stage(c, c->d_q[c->cur], c->d_q[1 - c->cur], c->d_res, 1.0, 0.0, 0.0, true, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e != cudaSuccess && rc == DG_OK) rc = cuda_fail(c, e, "stage timing");
    (type == 0 ? *us_w : *us_t) = 1e3 * double(ms) / nrep;
  }
  c->m32 = m32;
  c->m64 = m64;
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (rc) return rc;
  return check_device_error(c);
}

int dg_set_launch_variant(dg_ctx* c, int variant) {
  if (!c) return DG_ERR_ARG;
  const int bpc = (variant >> 1) & 3;
  const bool onthefly = (variant & 1) != 0, split = (variant & 8) != 0;
  // bits: 0 factor recomputed, 1-2 blocks per CTA (1 or 2), 3 split stage
  if ((variant & ~15) != 0 || bpc < 1 || bpc > 2 || (bpc == 2 && !(c->prec == DG_F32 && c->N == 3)))
    return c->fail(DG_ERR_ARG, "unknown launch variant");
  if (split && (onthefly || bpc != 1 || c->prec != DG_F32 || c->mass != DG_MASS_STORED || c->op != DG_OPS_FP32))
    return c->fail(DG_ERR_ARG, "the split stage needs FP32 fields and applies, the stored factor, one block per CTA");
  c->tuned_bpc = bpc;
  c->tuned_onthefly = onthefly && c->mass == DG_MASS_STORED;
  c->tuned_split = split ? 1 : -1;
  drop_graphs(c);
  return DG_OK;
}

namespace {
// Rebuild and upload the bound context's mesh tables for its current shot
// group (the blob's size does not depend on it), zero the state buffers and
// the simulation time, and drop the captured step graphs.  Synchronous.
int relayout(dg_ctx* c) {
  const BlobLayout L = blob_layout(c);
  if (L.total != c->mesh_bytes) return c->fail(DG_ERR_STATE, "mesh blob size changed");
  std::vector<unsigned char> blob;
  if (c->prec == DG_F64) {
    fill_blob<double>(c, L, blob);
    fill_devmesh<double>(c, L, c->m64);
  } else {
    fill_blob<float>(c, L, blob);
    fill_devmesh<float>(c, L, c->m32);
  }
  c->tri_far = triangle_neighbours_far(blob, L.w_nbr, L.w_code, vKw(c));
  drop_graphs(c);
  cudaError_t e = cudaMemcpyAsync(c->d_mesh, blob.data(), blob.size(), cudaMemcpyHostToDevice, c->stream);
  for (void* p : {c->d_q[0], c->d_q[1], c->d_res})
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, c->field_bytes, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "mesh re-layout");
  c->cur = 0;
  c->t = 0.0;
  return DG_OK;
}
}  // namespace

int dg_autotune_layout(dg_ctx* c, int nrep, int64_t* group, double* us) {
  if (!c) return DG_ERR_ARG;
  if (nrep < 1 || !group || !us) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_autotune_layout before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  // candidates: 1, 2, 4, ... and the shot count itself, each dividing it
  std::vector<int64_t> cand;
  for (int64_t g = 1; g <= c->shots; g *= 2)
    if (c->shots % g == 0) cand.push_back(g);
  if (cand.back() != c->shots) cand.push_back(c->shots);
  double best = 0.0;
  int64_t bestg = c->group();
  bool have = false;
  for (int64_t g : cand) {
    c->shot_group = g;
    int rc = relayout(c);
    double tw = 0.0, tt = 0.0;
    if (rc == DG_OK) rc = dg_stage_times(c, nrep, &tw, &tt);
    if (rc != DG_OK) {
      c->shot_group = bestg;
      relayout(c);
      return rc;
    }
    if (!have || tw + tt < best) {
      best = tw + tt;
      bestg = g;
      have = true;
    }
  }
  c->shot_group = bestg;
  const int rc = relayout(c);
  if (rc) return rc;
  *group = bestg;
  *us = best;
  return DG_OK;
}

int dg_autotune(dg_ctx* c, int nrep, int* variant, double* us) {
  if (!c) return DG_ERR_ARG;
  if (nrep < 1 || !variant || !us) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_autotune before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  // candidates: (factor recomputed in the stage?, wedge blocks per CTA, split over field pairs)
  struct Cand {
    bool onthefly;
    int bpc, split;
  };
  std::vector<Cand> cand;
  const int maxb = (c->prec == DG_F32 && c->N == 3) ? 2 : 1;
  for (int onthefly = 0; onthefly < 2; ++onthefly) {
    if (!onthefly && c->mass != DG_MASS_STORED) continue;
    for (int b = 1; b <= maxb; ++b) cand.push_back({onthefly != 0, b, -1});
  }
  // the field-pair split kernel: FP32 CUDA-core applies with the stored factor
  if (c->prec == DG_F32 && c->mass == DG_MASS_STORED && c->op == DG_OPS_FP32) cand.push_back({false, 1, 1});
  double best = 0.0;
  int besti = -1;
  for (size_t i = 0; i < cand.size(); ++i) {
    c->tuned_onthefly = cand[i].onthefly;
    c->tuned_bpc = cand[i].bpc;
    c->tuned_split = cand[i].split;
    double tw = 0.0, tt = 0.0;
    const int rc = dg_stage_times(c, nrep, &tw, &tt);
    if (rc) {
      c->tuned_onthefly = false;
      c->tuned_bpc = 0;
      c->tuned_split = 0;
      return rc;
    }
    if (besti < 0 || tw < best) {
      best = tw;
      besti = int(i);
    }
  }
  c->tuned_onthefly = cand[besti].onthefly;
  c->tuned_bpc = cand[besti].bpc;
  c->tuned_split = cand[besti].split;
  // captured step graphs hold the previous launch shape: capture again on the next step
  for (int p = 0; p < 2; ++p)
    if (c->gexec[p]) {
      cudaGraphExecDestroy(c->gexec[p]);
      c->gexec[p] = nullptr;
    }
  *variant = (cand[besti].bpc << 1) | (cand[besti].onthefly ? 1 : 0) | (cand[besti].split > 0 ? 8 : 0);
  *us = best;
  return DG_OK;
}

// ------------------------------------------------------------ receivers, adjoint
namespace {
constexpr int kAdjFields = 14;
enum { kAdjMuq = 0, kAdjX0 = 1, kAdjX1 = 2, kAdjRes = 3, kAdjQs = 4 /*4 buffers*/, kAdjScr = 8, kAdjRs = 9 /*5*/ };
// FP64 gradient sums per device element: [d/dkappa wedges][d/drho wedges][d/dkappa tets][d/drho tets]
size_t adj_grad_bytes(const dg_ctx* c) { return align256(size_t(nblk(vKw(c))) * kB * sizeof(double)); }
size_t adj_tgrad_bytes(const dg_ctx* c) { return align256(size_t(nblk(vKt(c))) * kB * sizeof(double)); }
void* adj_field(dg_ctx* c, int i) { return c->adj + size_t(i) * c->field_bytes; }
double* adj_gk(dg_ctx* c) { return reinterpret_cast<double*>(c->adj + kAdjFields * c->field_bytes); }
double* adj_gr(dg_ctx* c) { return reinterpret_cast<double*>(c->adj + kAdjFields * c->field_bytes + adj_grad_bytes(c)); }
double* adj_tgk(dg_ctx* c) {
  return reinterpret_cast<double*>(c->adj + kAdjFields * c->field_bytes + 2 * adj_grad_bytes(c));
}
double* adj_tgr(dg_ctx* c) {
  return reinterpret_cast<double*>(c->adj + kAdjFields * c->field_bytes + 2 * adj_grad_bytes(c) + adj_tgrad_bytes(c));
}
// FP64 face sums of the wedges, [face 0..4][device wedge]: dt times the penalty
// derivative of each face, written by the face's owner for both of its elements
double* adj_gz(dg_ctx* c) {
  return reinterpret_cast<double*>(c->adj + kAdjFields * c->field_bytes + 2 * adj_grad_bytes(c) + 2 * adj_tgrad_bytes(c));
}
}  // namespace

int dg_sample(dg_ctx* c, void* d_out) {
  if (!c) return DG_ERR_ARG;
  if (!d_out) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_sample before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc) return rc;
  if (c->prec == DG_F64)
    rc = sample_f64(c->N, c->m64, static_cast<const double*>(c->d_q[c->cur]), static_cast<double*>(d_out),
                    int(c->shots), c->stream);
  else
    rc = sample_f32(c->N, c->m32, static_cast<const float*>(c->d_q[c->cur]), static_cast<float*>(d_out),
                    int(c->shots), c->stream);
  if (rc) return cuda_fail(c, cudaError_t(rc), "sample launch");
  return DG_OK;
}

int dg_save_state(dg_ctx* c, void* d_dst) {
  if (!c) return DG_ERR_ARG;
  if (!d_dst) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_save_state before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  cudaError_t e = cudaMemcpyAsync(d_dst, c->d_q[c->cur], c->field_bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "state save");
  return DG_OK;
}

int dg_load_state(dg_ctx* c, const void* d_src, double t) {
  if (!c) return DG_ERR_ARG;
  if (!d_src || !std::isfinite(t)) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_load_state before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  cudaError_t e = cudaMemcpyAsync(c->d_q[c->cur], d_src, c->field_bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "state load");
  c->t = t;
  // the clock by a one-thread kernel on the stream: the call stays asynchronous
  const int rc = c->prec == DG_F64 ? set_clock_f64(c->N, c->m64.clock, t, c->stream)
                                   : set_clock_f32(c->N, c->m32.clock, t, c->stream);
  if (rc) return cuda_fail(c, cudaError_t(rc), "clock set");
  return DG_OK;
}

int dg_adjoint_bytes(const dg_ctx* c, size_t* bytes) {
  if (!c) return DG_ERR_ARG;
  if (!bytes) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->N) return c->fail(DG_ERR_STATE, "call needs dg_set_order first");
  *bytes = kAdjFields * field_bytes_of(c) + 7 * adj_grad_bytes(c) + 2 * adj_tgrad_bytes(c);
  return DG_OK;
}

int dg_adjoint_bind(dg_ctx* c, void* d_work) {
  if (!c) return DG_ERR_ARG;
  if (!d_work) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_adjoint_bind before dg_bind");
  if (c->N == 5 && c->prec == DG_F64)
    return c->fail(DG_ERR_ORDER, "the adjoint at N = 5 needs DG_F32 (the FP64 gradient kernel exceeds shared memory)");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  if (!c->grad_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&c->grad_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_gfork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_gjoin, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(c, e, "gradient stream");
  }
  c->adj = static_cast<unsigned char*>(d_work);
  return dg_adjoint_reset(c);
}

int dg_adjoint_reset(dg_ctx* c) {
  if (!c) return DG_ERR_ARG;
  if (!c->adj) return c->fail(DG_ERR_STATE, "dg_adjoint_reset before dg_adjoint_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  size_t bytes = 0;
  dg_adjoint_bytes(c, &bytes);
  cudaError_t e = cudaMemsetAsync(c->adj, 0, bytes, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint reset");
  c->adj_x = kAdjX0;
  return DG_OK;
}

int dg_adjoint_inject(dg_ctx* c, const void* d_resid) {
  if (!c) return DG_ERR_ARG;
  if (!d_resid) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->adj) return c->fail(DG_ERR_STATE, "dg_adjoint_inject before dg_adjoint_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc) return rc;
  if (c->prec == DG_F64)
    rc = inject_f64(c->N, c->m64, static_cast<double*>(adj_field(c, kAdjMuq)), static_cast<double*>(adj_field(c, c->adj_x)),
                    static_cast<const double*>(d_resid), int(c->shots), kLSRK_B[4], c->stream);
  else
    rc = inject_f32(c->N, c->m32, static_cast<float*>(adj_field(c, kAdjMuq)), static_cast<float*>(adj_field(c, c->adj_x)),
                    static_cast<const float*>(d_resid), int(c->shots), float(kLSRK_B[4]), c->stream);
  if (rc) return cuda_fail(c, cudaError_t(rc), "adjoint inject launch");
  return DG_OK;
}

namespace {
// the five adjoint stages of one step in reverse (variables mu = P W^{-1} lambda):
// gradient terms of stage s with x = mu_K, then mu_Q += dt A x and x <- a_s x +
// b_{s-1} mu_Q.  Q[s] is the input of forward stage s (Q[0] = q_n), R[s] its
// right-hand side.
int adjoint_reverse_stages(dg_ctx* c, double dt, const void* const* Q, const void* const* R) {
  int rc = DG_OK;
  for (int st = 4; st >= 0 && rc == DG_OK; --st) {
    void* xin = adj_field(c, c->adj_x);
    void* xout = adj_field(c, c->adj_x == kAdjX0 ? kAdjX1 : kAdjX0);
    // the gradient terms of stage st read x (= xin), Q[st] and R[st]; the
    // adjoint stage reads xin and writes xout and mu_Q: the two run side by
    // side, the gradient on its own stream, joined before the next stage
    // overwrites xin
    cudaStream_t gs = c->grad_stream ? c->grad_stream : c->stream;
    if (gs != c->stream) {
      cudaError_t e = cudaEventRecord(c->ev_gfork, c->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(gs, c->ev_gfork, 0);
      if (e != cudaSuccess) return cuda_fail(c, e, "gradient fork");
    }
    int lr;
    if (c->prec == DG_F64)
      lr = grad_f64(c->N, c->m64, static_cast<const double*>(xin), static_cast<const double*>(Q[st]),
                    static_cast<const double*>(R[st]), dt, c->flux, c->bc, adj_gk(c), adj_gr(c), adj_gz(c), gs);
    else
      lr = grad_f32(c->N, c->m32, static_cast<const float*>(xin), static_cast<const float*>(Q[st]),
                    static_cast<const float*>(R[st]), dt, c->flux, c->bc, adj_gk(c), adj_gr(c), adj_gz(c), gs);
    if (lr) return cuda_fail(c, cudaError_t(lr), "gradient launch");
    if (c->prec == DG_F64)
      lr = tgrad_f64(c->N, c->m64, static_cast<const double*>(xin), static_cast<const double*>(Q[st]),
                     static_cast<const double*>(R[st]), dt, c->flux, c->bc, adj_tgk(c), adj_tgr(c), gs);
    else
      lr = tgrad_f32(c->N, c->m32, static_cast<const float*>(xin), static_cast<const float*>(Q[st]),
                     static_cast<const float*>(R[st]), dt, c->flux, c->bc, adj_tgk(c), adj_tgr(c), gs);
    if (lr) return cuda_fail(c, cudaError_t(lr), "tet gradient launch");
    StageExtra x;
    x.g = kLSRK_A[st];
    x.no_sources = true;
    rc = launch_stage(c, xin, xout, adj_field(c, kAdjMuq), 1.0, kLSRK_B[(st + 4) % 5], dt, true, c->stream, 0.0, x);
    if (gs != c->stream) {
      cudaError_t e = cudaEventRecord(c->ev_gjoin, gs);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_gjoin, 0);
      if (e != cudaSuccess && rc == DG_OK) rc = cuda_fail(c, e, "gradient join");
    }
    c->adj_x = c->adj_x == kAdjX0 ? kAdjX1 : kAdjX0;
  }
  return rc;
}

constexpr int kRecFields = 10;  // q_n, Q_1..Q_4, r_1..r_5
}  // namespace

int dg_adjoint_step(dg_ctx* c, double dt) {
  if (!c) return DG_ERR_ARG;
  if (!(dt > 0)) return c->fail(DG_ERR_ARG, "dt must be positive");
  if (!c->adj) return c->fail(DG_ERR_STATE, "dg_adjoint_step before dg_adjoint_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc) return rc;
  // the forward step from the current state and time, keeping every stage's
  // input Q_{s-1} and right-hand side r_s = A Q_{s-1} + f(t + c_s dt)
  const void* Q[5] = {c->d_q[c->cur], adj_field(c, kAdjQs), adj_field(c, kAdjQs + 1), adj_field(c, kAdjQs + 2),
                      adj_field(c, kAdjQs + 3)};
  const void* R[5];
  for (int st = 0; st < 5 && rc == DG_OK; ++st) {
    void* qout = adj_field(c, st < 4 ? kAdjQs + st : kAdjScr);
    StageExtra x;
    x.rhs_out = adj_field(c, kAdjRs + st);
    R[st] = x.rhs_out;
    rc = launch_stage(c, Q[st], qout, adj_field(c, kAdjRes), kLSRK_A[st], kLSRK_B[st], dt, true, c->stream, kLSRK_C[st], x);
  }
  if (rc) return rc;
  return adjoint_reverse_stages(c, dt, Q, R);
}

int dg_step_record_bytes(const dg_ctx* c, size_t* bytes) {
  if (!c) return DG_ERR_ARG;
  if (!bytes) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->N) return c->fail(DG_ERR_STATE, "call needs dg_set_order first");
  *bytes = kRecFields * field_bytes_of(c);
  return DG_OK;
}

int dg_step_record_chain(dg_ctx* c, double dt, int64_t nsteps, void* const* d_recs) {
  if (!c) return DG_ERR_ARG;
  if (nsteps < 0 || (nsteps > 0 && !d_recs)) return c->fail(DG_ERR_ARG, "null or invalid argument");
  for (int64_t i = 0; i < nsteps; ++i)
    if (!d_recs[i] || reinterpret_cast<uintptr_t>(d_recs[i]) % 256) return c->fail(DG_ERR_ARG, "null or misaligned record");
  if (!(dt > 0)) return c->fail(DG_ERR_ARG, "dt must be positive");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_step_record before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc || nsteps == 0) return rc;
  const size_t fb = c->field_bytes;
  // record i: slot 0 takes q_i, the stages run slot s -> slot s + 1, and the last
  // one writes slot 0 of record i + 1 (the bound buffer after the last step):
  // the same launches as captured steps, one state copy per chain
  cudaError_t e = cudaMemcpyAsync(d_recs[0], c->d_q[c->cur], fb, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "record copy");
  double* clk = (c->prec == DG_F64) ? c->m64.clock : c->m32.clock;
  for (int64_t i = 0; i < nsteps; ++i) {
    unsigned char* rec = static_cast<unsigned char*>(d_recs[i]);
    for (int st = 0; st < 5 && rc == DG_OK; ++st) {
      StageExtra x;
      x.rhs_out = rec + size_t(5 + st) * fb;
      void* qout = st < 4 ? static_cast<void*>(rec + size_t(st + 1) * fb)
                          : (i + 1 < nsteps ? d_recs[i + 1] : c->d_q[c->cur]);
      rc = launch_stage(c, rec + size_t(st) * fb, qout, c->d_res, kLSRK_A[st], kLSRK_B[st], dt, true, c->stream,
                        kLSRK_C[st], x);
    }
    if (rc) return rc;
    const int crc = (c->prec == DG_F64) ? clock_f64(c->N, clk, dt, c->stream) : clock_f32(c->N, clk, dt, c->stream);
    if (crc) return cuda_fail(c, cudaError_t(crc), "clock launch");
    c->t += dt;
  }
  return DG_OK;
}

int dg_step_record(dg_ctx* c, double dt, void* d_rec) {
  if (!c) return DG_ERR_ARG;
  if (!d_rec) return c->fail(DG_ERR_ARG, "null or misaligned record");
  void* recs[1] = {d_rec};
  return dg_step_record_chain(c, dt, 1, recs);
}

int dg_adjoint_step_recorded(dg_ctx* c, double dt, const void* d_rec) {
  if (!c) return DG_ERR_ARG;
  if (!d_rec || reinterpret_cast<uintptr_t>(d_rec) % 256) return c->fail(DG_ERR_ARG, "null or misaligned record");
  if (!(dt > 0)) return c->fail(DG_ERR_ARG, "dt must be positive");
  if (!c->adj) return c->fail(DG_ERR_STATE, "dg_adjoint_step_recorded before dg_adjoint_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc) return rc;
  const unsigned char* rec = static_cast<const unsigned char*>(d_rec);
  const size_t fb = c->field_bytes;
  const void* Q[5];
  const void* R[5];
  for (int st = 0; st < 5; ++st) {
    Q[st] = rec + size_t(st) * fb;
    R[st] = rec + size_t(5 + st) * fb;
  }
  return adjoint_reverse_stages(c, dt, Q, R);
}

int dg_adjoint_set(dg_ctx* c, const void* mu_q, const void* x, int on_device) {
  if (!c) return DG_ERR_ARG;
  if (!mu_q || !x) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->adj) return c->fail(DG_ERR_STATE, "dg_adjoint_set before dg_adjoint_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc) return rc;
  const size_t rs = c->prec == DG_F64 ? 8 : 4;
  const size_t bytes = size_t(4) * c->shots * (c->wedge_nodes + c->tet_nodes) * rs;
  const void* src[2] = {mu_q, x};
  void* dst[2] = {adj_field(c, kAdjMuq), adj_field(c, c->adj_x)};
  for (int i = 0; i < 2; ++i) {
    const void* from = src[i];
    if (!on_device) {
      cudaError_t e = cudaMemcpyAsync(adj_field(c, kAdjScr), src[i], bytes, cudaMemcpyHostToDevice, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "adjoint upload");
      from = adj_field(c, kAdjScr);
    }
    rc = launch_pack(c, from, dst[i], false, c->stream);
    if (rc) return rc;
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint upload");
  return DG_OK;
}

int dg_adjoint_get(dg_ctx* c, void* dst, int on_device) {
  if (!c) return DG_ERR_ARG;
  if (!dst) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->adj) return c->fail(DG_ERR_STATE, "dg_adjoint_get before dg_adjoint_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc) return rc;
  const size_t rs = c->prec == DG_F64 ? 8 : 4;
  const size_t bytes = size_t(4) * c->shots * (c->wedge_nodes + c->tet_nodes) * rs;
  void* out = on_device ? dst : adj_field(c, kAdjScr);
  rc = launch_pack(c, out, adj_field(c, kAdjMuq), true, c->stream);
  if (rc) return rc;
  if (!on_device) {
    cudaError_t e = cudaMemcpyAsync(dst, out, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "adjoint download");
  }
  return DG_OK;
}

int dg_adjoint_gradient(dg_ctx* c, double* g_kappa, double* g_rho) {
  if (!c) return DG_ERR_ARG;
  if (!g_kappa || !g_rho) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->adj) return c->fail(DG_ERR_STATE, "dg_adjoint_gradient before dg_adjoint_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  const int64_t Kw = int64_t(c->wedges.size()), nv = nblk(vKw(c)) * kB;
  const int64_t Kt = int64_t(c->tets.size()), nt = nblk(vKt(c)) * kB;
  std::vector<double> gk(nv), gr(nv), gz(5 * nv), tk(nt), tr(nt);
  cudaError_t e = cudaMemcpyAsync(gk.data(), adj_gk(c), nv * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gr.data(), adj_gr(c), nv * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(gz.data(), adj_gz(c), 5 * nv * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && nt > 0)
    e = cudaMemcpyAsync(tk.data(), adj_tgk(c), nt * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && nt > 0)
    e = cudaMemcpyAsync(tr.data(), adj_tgr(c), nt * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "gradient download");
  for (int64_t k = 0; k < c->K; ++k) g_kappa[k] = g_rho[k] = 0.0;
  // sum over shots in shot order, per element of either type; a wedge's face
  // sums G (dt times dJ/dz through the penalty) enter through z = rho c:
  // dz/dkappa = 1 / (2 c), dz/drho = c / 2
  for (int64_t s = 0; s < c->shots; ++s) {
    for (int64_t w = 0; w < Kw; ++w) {
      const int64_t v = shot_vid(s, w, Kw, c->group());
      const int64_t k = c->wedges[w];
      double G = 0.0;
      for (int f = 0; f < 5; ++f) G += gz[f * nv + v];
      const double cc = std::sqrt(c->c2[k]);
      g_kappa[k] += gk[v] + G / (2.0 * cc);
      g_rho[k] += gr[v] + G * (0.5 * cc);
    }
    for (int64_t t = 0; t < Kt; ++t) {
      const int64_t v = shot_vid(s, t, Kt, c->group());
      g_kappa[c->tets[t]] += tk[v];
      g_rho[c->tets[t]] += tr[v];
    }
  }
  return check_device_error(c);
}

int dg_energy(dg_ctx* c, double* E) {
  if (!c) return DG_ERR_ARG;
  if (!E) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_energy before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int rc = ensure_ops(c);
  if (rc) return rc;
  int lr;
  double* dE;
  if (c->prec == DG_F64) {
    lr = energy_f64(c->N, c->m64, static_cast<const double*>(c->d_q[c->cur]), c->stream);
    dE = c->m64.energy;
  } else {
    lr = energy_f32(c->N, c->m32, static_cast<const float*>(c->d_q[c->cur]), c->stream);
    dE = c->m32.energy;
  }
  if (lr) return cuda_fail(c, cudaError_t(lr), "energy launch");
  cudaError_t e = cudaMemcpyAsync(E, dE, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "energy download");
  return check_device_error(c);
}

int dg_energy_static(dg_ctx* c, const void* d_q, double* E) {
  if (!c) return DG_ERR_ARG;
  if (!d_q || !E) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_energy_static before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  const int64_t K = vKw(c) + vKt(c);
  const int64_t nblocks = (K + 127) / 128;
  if (nblocks > kStaticPartials)
    return c->fail(DG_ERR_ARG, "dg_energy_static supports at most " + std::to_string(int64_t(kStaticPartials) * 128) +
                                   " elements");
  double* scratch = nullptr;
  int rc = energy_static_scratch(c->device, &scratch);
  if (rc) return cuda_fail(c, cudaError_t(rc), "static scratch address");
  const unsigned char* blob = static_cast<const unsigned char*>(c->d_mesh);
  if (c->prec == DG_F64)
    rc = launch_energy_static<double>(c->N, c->m64, static_cast<const double*>(d_q),
                                      reinterpret_cast<const double*>(blob + c->wops_off), scratch, int(nblocks), c->stream);
  else
    rc = launch_energy_static<float>(c->N, c->m32, static_cast<const float*>(d_q),
                                     reinterpret_cast<const float*>(blob + c->wops_off), scratch, int(nblocks), c->stream);
  if (rc) return cuda_fail(c, cudaError_t(rc), "static energy launch");
  cudaError_t e = cudaMemcpyAsync(E, scratch + kStaticPartials, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "static energy download");
  if (!std::isfinite(*E)) return c->fail(DG_ERR_NONFINITE, "non-finite energy");
  // a device-side error raised by earlier work on the stream (bounded waits)
  return check_device_error(c);
}

int dg_expire_wait(dg_ctx* c) {
  if (!c) return DG_ERR_ARG;
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_expire_wait before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  int* derr = (c->prec == DG_F64) ? c->m64.err : c->m32.err;
  const int rc = (c->prec == DG_F64) ? wait_expire_f64(c->N, derr, c->stream) : wait_expire_f32(c->N, derr, c->stream);
  if (rc) return cuda_fail(c, cudaError_t(rc), "wait-expiry launch");
  return DG_OK;
}

int dg_sync(dg_ctx* c) {
  if (!c) return DG_ERR_ARG;
  if (!c->bound) return c->fail(DG_ERR_STATE, "dg_sync before dg_bind");
  DeviceGuard device_guard(c);
  if (device_guard.err != cudaSuccess) return cuda_fail(c, device_guard.err, "set device");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  return check_device_error(c);
}

int dg_time(const dg_ctx* c, double* t) {
  if (!c) return DG_ERR_ARG;
  if (!t) return c->fail(DG_ERR_ARG, "null or invalid argument");
  *t = c->t;
  return DG_OK;
}

int dg_stable_dt(const dg_ctx* c, double cfl, double* dt) {
  if (!c) return DG_ERR_ARG;
  if (!dt || !(cfl > 0)) return c->fail(DG_ERR_ARG, "null or invalid argument");
  if (!c->N) return c->fail(DG_ERR_STATE, "call needs dg_set_order first");
  double best = INFINITY;
  for (int64_t k = 0; k < c->K; ++k) {
    const double ratio = c->etype[k] == DG_WEDGE ? wedge_stable_ratio(c, k) : tet_stable_ratio(c, k);
    const double cc = std::sqrt(c->c2[k]);
    best = std::min(best, 1.0 / (cc * (c->N + 1) * (c->N + 1) * ratio));
  }
  *dt = cfl * best;
  return DG_OK;
}

const char* dg_last_error(const dg_ctx* c) { return c ? c->err.c_str() : "null context"; }

void dg_destroy(dg_ctx* c) {
  if (!c) return;
  DeviceGuard device_guard(c);
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->tet_stream) cudaStreamDestroy(c->tet_stream);
  if (c->grad_stream) cudaStreamDestroy(c->grad_stream);
  if (c->ev_gfork) cudaEventDestroy(c->ev_gfork);
  if (c->ev_gjoin) cudaEventDestroy(c->ev_gjoin);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  delete c;
}

}  // extern "C"
