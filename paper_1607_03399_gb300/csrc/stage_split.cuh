// Wedge stage with each (element, slice) split over two threads by field
// pairs (included by kernels.cuh after k_wedge_stage, whose helpers it uses).
//
// Same operator as k_wedge_stage (Sections 3.2, 4.2; fused LSRK update), for
// the stored mass factor.  A CTA holds one 32-wedge block with 2 (N+1)
// warps: warp 2 j + h owns GLL slice j and the field pair h -- h = 0 the
// pressure and u_x, h = 1 u_y and u_z (fields (0, 1) and (2, 3) of a node
// record, so the update moves 8-byte pairs).  Each thread keeps the
// weak-form accumulators of two fields only (2 Nt instead of 4 Nt), so twice
// the warps can be resident where the one-thread-per-slice kernel is limited
// by registers (N = 4).  A launch variant of dg_autotune: at N = 4 on the
// 524,288-wedge workload, both on packed pairs, it measured 1248 us per stage
// against 1061 us for the one-thread form (96 registers with spills, duplicated
// face gathers; the one-thread form has since staged its residual slab too,
// 810 us), so it is not the default.  Work split:
//   fluxes: both halves form the quadrilateral-face jumps of their slice
//     (the same neighbour traces); h = 0 lifts F_p and n_x F_u, h = 1 n_y F_u;
//     the triangle-face node fluxes are spread over all warps;
//   weak part: h = 0 builds G_p (D_t of u_x, u_y, u_z) and G_ux (D_t p),
//     h = 1 G_uy and G_uz (D_t p); each applies M^tri to its two vectors and
//     solves with the factor for its two right-hand sides;
//   strong part: h = 0 forms div u = D_r (r.u) + D_s (s.u), h = 1 forms
//     D_r p and D_s p, hence d_x p (handed to h = 0 through shared memory and
//     a barrier of the slice's two warps) and d_y p;
//   update: each half its two fields.
#pragma once

namespace dgw {
namespace REALNS {

template <int N>
struct SplitSmem {
  static constexpr int Nt = nt_of(N), Nq = N + 1, Np = Nt * Nq;
  static constexpr int q = 0;                          // [Np][32][4] state slab
  static constexpr int L = q + 4 * Np * kB;            // [NL4][32][4] mass factor
  static constexpr int F = L + nl4_of(N) * 4 * kB;     // [4][Nt][32] triangle-face fluxes
  static constexpr int G = F + 4 * Nt * kB;            // [G_STAGE][32] geometry
  static constexpr int X = G + G_STAGE * kB;           // [Nq][Nt][32] d_x p, handed from h = 1 to h = 0
  static constexpr int reals = X + Nq * Nt * kB;
};
template <int N>
__host__ __device__ constexpr int split_smem_bytes() {
  return 32 + SplitSmem<N>::reals * int(sizeof(real));
}

template <int N>
__global__ void __launch_bounds__(64 * (N + 1), 2) k_wedge_stage_split(const StageArgs<real> A, bool rk) {
  constexpr int Nt = nt_of(N), Nq = N + 1, Np = Nt * Nq;
  using SM = SplitSmem<N>;
  const AllOps<N, real>& O = OPS<N>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, j = w >> 1, h = w & 1;
  const int lane = threadIdx.x & 31;
  const bool leader = threadIdx.x == 0;
  // [0] state slab and factor, [1] unused, [2] vertex coordinates
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  int* status = reinterpret_cast<int*>(smem_raw + 24);
  real* base = reinterpret_cast<real*>(smem_raw + 32);
  real* sq = base + SM::q;
  real* sL = base + SM::L;
  real* sF = base + SM::F;
  real* sG = base + SM::G;
  real* sX = base + SM::X;
  const DevMesh<real>& M = A.m;
  const real* __restrict__ qin = A.q_in;
  real* __restrict__ qout = A.q_out;
  real* __restrict__ resg = A.res;
  const int blk = blockIdx.x;
  const int e = blk * kB + lane;
  const int Kp = M.Kw_pad;
  constexpr int NL4 = nl4_of(N);
  constexpr uint32_t slab_bytes = uint32_t(4 * Np * kB * sizeof(real));
  constexpr uint32_t fac_bytes = uint32_t(NL4 * 4 * kB * sizeof(real));
  constexpr uint32_t xyz_bytes = uint32_t(12 * kB * sizeof(real));
#define GEO(item) sG[(item) * kB + lane]
  auto block_sync = [&]() { asm volatile("bar.sync 1, %0;" ::"n"(64 * Nq) : "memory"); };
  // the two warps of slice j (named barriers 2 .. Nq + 1, immediate ids)
  auto pair_sync = [&]() {
    static_assert(N + 1 <= 6, "at most six slices");
    switch (j) {
      case 0: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
      case 1: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
      case 2: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
      case 3: asm volatile("bar.sync 5, 64;" ::: "memory"); break;
      case 4: asm volatile("bar.sync 6, 64;" ::: "memory"); break;
      default: asm volatile("bar.sync 7, 64;" ::: "memory"); break;
    }
  };

  if (leader) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[2], 1);
    fence_mbar_init();
    mbar_expect_tx(&bar[2], xyz_bytes);
    bulk_g2s(sG, M.w_xyz + int64_t(blk) * 12 * kB, xyz_bytes, &bar[2]);
    mbar_expect_tx(&bar[0], slab_bytes + fac_bytes);
    bulk_g2s(sq, qin + int64_t(blk) * 4 * Np * kB, slab_bytes, &bar[0]);
    bulk_g2s(sL, M.w_fac + int64_t(blk) * NL4 * 4 * kB, fac_bytes, &bar[0]);
  }
  // face neighbours, their impedances and the source flag while the slabs fly
  const real zM = M.w_mat[2 * Kp + e];
  int qnbr[3], qcode[3];
  real zPq[3];
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) {
    qnbr[ed] = M.w_nbr[(2 + ed) * Kp + e];
    qcode[ed] = M.w_code[(2 + ed) * Kp + e];
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
  const bool src = h == 0 && M.nsrc > 0 && has_source(M, 6, e);
  bool geo_ok = true;
  __syncwarp();
  if (w == 0) {
    geo_ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bar[2], 0));
    if (geo_ok) wedge_geometry<G_STAGE>(sG, lane);
  }
  if (leader) *status = (mbar_wait_bounded(&bar[0], 0) && geo_ok) ? 1 : 0;
  block_sync();
  if (*reinterpret_cast<volatile int*>(status) == 0) {
    if (leader) {
      atomicOr(M.err, kErrTimeout);
      mbar_wait_bounded(&bar[0], 0);
      mbar_wait_bounded(&bar[2], 0);
    }
    return;
  }

  // 1. prologue: quadrilateral-face fluxes of slice j lifted into this
  //    half's accumulators (a: p or u_y, b: u_x or u_z); the triangle-face
  //    node fluxes spread over all warps
  // accumulators of node i as one packed pair: (p, u_x) for h = 0, (u_y, u_z) for h = 1
  constexpr int NH = (Nt + 1) / 2;
  real2 W[Nt];
#pragma unroll
  for (int i = 0; i < Nt; ++i) W[i] = dup2(real(0));
#pragma unroll
  for (int ed = 0; ed < 3; ++ed) {
    const int nbr = qnbr[ed];
    const bool bnd = nbr < 0;
    const bool inblk = bnd || (nbr >> 5) == blk;
    const int ep = bnd ? ed : qcode[ed] >> 1, rev = bnd ? 0 : qcode[ed] & 1;
    Q4 nv[Nq];
    if (inblk) {
      const int nl = bnd ? lane : (nbr & 31);
#pragma unroll
      for (int m = 0; m < Nq; ++m) nv[m] = lds4(sq, j * Nt + O.tab.edge[ep][rev ? N - m : m], nl);
    } else {
      const real* gb = qin + widx<N>(nbr >> 5, 0, nbr & 31);
#pragma unroll
      for (int m = 0; m < Nq; ++m) nv[m] = ldg4(gb, int64_t(j * Nt + O.tab.edge[ep][rev ? N - m : m]) * (kB * 4));
    }
    const real nx = GEO(G_QNX0 + ed), ny = GEO(G_QNY0 + ed);
    real Fp[Nq], Fu[Nq];
    real tau_p, tau_u;
    taus(A.flux, zM, zPq[ed], tau_p, tau_u);
#pragma unroll
    for (int m = 0; m < Nq; ++m) {
      const Q4 o = lds4(sq, j * Nt + edge_node(N, ed, m), lane);
      real bdp, bdun;
      boundary_jumps(A.bc, o.p, nx * o.u + ny * o.v, bdp, bdun);
      const real dp = bnd ? bdp : nv[m].p - o.p;
      const real dun = bnd ? bdun : nx * (nv[m].u - o.u) + ny * (nv[m].v - o.v);
      penalty_flux(dp, dun, tau_p, tau_u, Fp[m], Fu[m]);
    }
    // W += M~_e F, M~_e = (L_e/4)(h_a Mea + h_b Meb) along the edge, identity in t
    // (Mea, Meb by output pairs)
    const real ca = GEO(G_QCA0 + ed), cbq = GEO(G_QCB0 + ed);
    constexpr int NQH = (Nq + 1) / 2;
    real2 gua[NQH], gub[NQH], gpa[NQH], gpb[NQH];
#pragma unroll
    for (int hh = 0; hh < NQH; ++hh) gua[hh] = gub[hh] = gpa[hh] = gpb[hh] = dup2(real(0));
#pragma unroll
    for (int n = 0; n < Nq; ++n) {
      const real2 fu2 = dup2(Fu[n]), fp2 = dup2(Fp[n]);
#pragma unroll
      for (int hh = 0; hh < NQH; ++hh) {
        const real2 ea = cpair(O.w.MeaP, Nq, hh, n), eb = cpair(O.w.MebP, Nq, hh, n);
        gua[hh] = fma2(ea, fu2, gua[hh]);
        gub[hh] = fma2(eb, fu2, gub[hh]);
        if (h == 0) {
          gpa[hh] = fma2(ea, fp2, gpa[hh]);
          gpb[hh] = fma2(eb, fp2, gpb[hh]);
        }
      }
    }
#pragma unroll
    for (int m = 0; m < Nq; ++m) {
      const real gu = ca * pair_row(gua, m) + cbq * pair_row(gub, m);
      const int i = edge_node(N, ed, m);
      if (h == 0) {
        W[i].x += ca * pair_row(gpa, m) + cbq * pair_row(gpb, m);
        W[i].y += nx * gu;
      } else {
        W[i].x += ny * gu;
      }
    }
  }
  // triangle-face node fluxes (bottom then top), round-robin over all warps
#pragma unroll
  for (int t = 0; t < (2 * Nt + 2 * Nq - 1) / (2 * Nq); ++t) {
    const int idx = w + t * 2 * Nq;
    if (idx >= 2 * Nt) break;
    const int fb = idx >= Nt ? 1 : 0;
    const int k = idx - fb * Nt;
    const real nn0 = GEO(fb ? G_NT0 : G_NB0), nn1 = GEO(fb ? G_NT1 : G_NB1), nn2 = GEO(fb ? G_NT2 : G_NB2);
    const int nbr = tnbr[fb];
    const int code = tcode[fb];
    const Q4 o = lds4(sq, (fb ? N * Nt : 0) + k, lane);
    const real unM = nn0 * o.u + nn1 * o.v + nn2 * o.w;
    real tau_p, tau_u, bdp, bdun;
    taus(A.flux, zM, fb ? zPt[1] : zPt[0], tau_p, tau_u);
    boundary_jumps(A.bc, o.p, unM, bdp, bdun);
    const bool bnd = nbr < 0;
    const bool ntet = !bnd && (code & kCodeTet) != 0;
    const int nf = bnd ? fb : (code >> 4) & 3;
    const int nk = bnd ? k : O.tab.tri_perm[code & 15][k];
    const int nbe = bnd ? e : nbr;
    const int node = ntet ? O.tab.tet_face[nf][nk] : (nf ? N * Nt : 0) + nk;
    const bool inblk = !ntet && (nbe >> 5) == blk;
    const Q4 nv = inblk ? lds4(sq, node, nbe & 31)
                        : ldg4(qin, ntet ? tidx<N>(M.tet_off, nbe >> 5, node, nbe & 31) : widx<N>(nbe >> 5, node, nbe & 31));
    const real dp = bnd ? bdp : nv.p - o.p;
    const real dun = bnd ? bdun : nn0 * nv.u + nn1 * nv.v + nn2 * nv.w - unM;
    real Fp, Fu;
    penalty_flux(dp, dun, tau_p, tau_u, Fp, Fu);
    sF[((2 * fb + 0) * Nt + k) * kB + lane] = Fp;
    sF[((2 * fb + 1) * Nt + k) * kB + lane] = Fu;
  }
  block_sync();

  // 2. weak part of slice j for this half's two fields: G -> M^tri G
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
    real Ga[Nt], Gb[Nt];
    if (h == 0) {
      const real nb0 = GEO(G_NB0) * cb, nt0 = GEO(G_NT0) * ct;
#pragma unroll
      for (int i = 0; i < Nt; ++i) {
        real2 dpu = dup2(real(0)), dvw = dup2(real(0));
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          const Q4 v = lds4(sq, m * Nt + i, lane);
          const real2 d2 = dup2(dtr[m]);
          dpu = fma2(d2, mk2(v.p, v.u), dpu);
          dvw = fma2(d2, mk2(v.v, v.w), dvw);
        }
        Ga[i] = cb * sF[(0 * Nt + i) * kB + lane] + ct * sF[(2 * Nt + i) * kB + lane] -
                (txJ * dpu.y + tyJ * dvw.x + Aj * dvw.y);
        Gb[i] = nb0 * sF[(1 * Nt + i) * kB + lane] + nt0 * sF[(3 * Nt + i) * kB + lane] - txJ * dpu.x;
      }
    } else {
      const real nb1 = GEO(G_NB1) * cb, nt1 = GEO(G_NT1) * ct, nb2 = GEO(G_NB2) * cb, nt2 = GEO(G_NT2) * ct;
#pragma unroll
      for (int i = 0; i < Nt; ++i) {
        real dpp = 0;
#pragma unroll
        for (int m = 0; m < Nq; ++m) dpp += dtr[m] * sq[((m * Nt + i) * kB + lane) * 4];
        const real f1 = sF[(1 * Nt + i) * kB + lane], f3 = sF[(3 * Nt + i) * kB + lane];
        Ga[i] = nb1 * f1 + nt1 * f3 - tyJ * dpp;
        Gb[i] = nb2 * f1 + nt2 * f3 - Aj * dpp;
      }
    }
    real2 aa[NH], ab[NH];
    apply_pairs<Nt, Nt>(O.w.MP, Ga, aa);
    apply_pairs<Nt, Nt>(O.w.MP, Gb, ab);
#pragma unroll
    for (int i = 0; i < Nt; ++i) W[i] = add2(W[i], mk2(pair_row(aa, i), pair_row(ab, i)));
  }
  // 3. X = (M^{tri,k})^{-1} W for the two right-hand sides: forward and
  //    backward sweeps over the packed factor, row by row
  {
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
      for (int k = 0; k < i; ++k) W[i] = fma2(dup2(-Lr[k]), W[k], W[i]);
      W[i] = mul2(W[i], dup2(Lr[i]));
    }
#pragma unroll
    for (int i = Nt - 1; i >= 0; --i) {
      real Lr[Nt];
      load_row(i, Lr);
      W[i] = mul2(W[i], dup2(Lr[i]));
#pragma unroll
      for (int k = 0; k < i; ++k) W[k] = fma2(dup2(-Lr[k]), W[i], W[k]);
    }
  }
  // 4. strong r, s parts (Lemma 3.1 metric terms): h = 0 div u, h = 1 D_r p,
  //    D_s p, whose d_x p goes to h = 0 through the slice's exchange table
  {
    const real rx = GEO(G_RX), ry = GEO(G_RY), sx = GEO(G_SX), sy = GEO(G_SY);
    // (D_r, D_s by output pairs, node l of the slice at a time)
    if (h == 0) {
      real2 dv[NH];
#pragma unroll
      for (int hh = 0; hh < NH; ++hh) dv[hh] = dup2(real(0));
#pragma unroll
      for (int l = 0; l < Nt; ++l) {
        const Q4 v = lds4(sq, j * Nt + l, lane);
        const real2 a2 = dup2(rx * v.u + ry * v.v), b2 = dup2(sx * v.u + sy * v.v);
#pragma unroll
        for (int hh = 0; hh < NH; ++hh) {
          dv[hh] = fma2(cpair(O.w.DrP, Nt, hh, l), a2, dv[hh]);
          dv[hh] = fma2(cpair(O.w.DsP, Nt, hh, l), b2, dv[hh]);
        }
      }
#pragma unroll
      for (int i = 0; i < Nt; ++i) W[i].x -= pair_row(dv, i);
      pair_sync();
#pragma unroll
      for (int i = 0; i < Nt; ++i) W[i].y -= sX[((j * Nt) + i) * kB + lane];
    } else {
      real2 pr[NH], ps[NH];
#pragma unroll
      for (int hh = 0; hh < NH; ++hh) pr[hh] = ps[hh] = dup2(real(0));
#pragma unroll
      for (int l = 0; l < Nt; ++l) {
        const real2 p2 = dup2(sq[(((j * Nt) + l) * kB + lane) * 4]);
#pragma unroll
        for (int hh = 0; hh < NH; ++hh) {
          pr[hh] = fma2(cpair(O.w.DrP, Nt, hh, l), p2, pr[hh]);
          ps[hh] = fma2(cpair(O.w.DsP, Nt, hh, l), p2, ps[hh]);
        }
      }
#pragma unroll
      for (int i = 0; i < Nt; ++i) {
        const real pri = pair_row(pr, i), psi = pair_row(ps, i);
        sX[((j * Nt) + i) * kB + lane] = rx * pri + sx * psi;
        W[i].x -= ry * pri + sy * psi;
      }
      pair_sync();
    }
  }

  // 5. point sources (pressure, h = 0) and the fused low-storage Runge-Kutta
  //    update (or the plain right-hand side) of this half's two fields
  const real kappa = M.w_mat[0 * Kp + e], irho = M.w_mat[1 * Kp + e];
  if (src) add_sources(M, 6, e, j * Nt, Np, *M.clock + A.c_stage * double(A.dt), W);
  const real2 sab = mk2(h == 0 ? kappa : irho, irho);
  if (e < M.Kw) {
#pragma unroll
    for (int i = 0; i < Nt; ++i) {
      const int n = j * Nt + i;
      const int64_t g = widx<N>(blk, n, lane) + 2 * h;
      const real2 r = mul2(W[i], sab);
      if (rk) {
        // res = a res + dt r, q = g q + b res on the packed pair
        const real2 r0 = *reinterpret_cast<const real2*>(resg + g);
        const real2 q0 = *reinterpret_cast<const real2*>(sq + (n * kB + lane) * 4 + 2 * h);
        const real2 rr = fma2(dup2(A.rk_a), r0, mul2(dup2(A.dt), r));
        const real2 qq = fma2(dup2(A.rk_g), q0, mul2(dup2(A.rk_b), rr));
        *reinterpret_cast<real2*>(resg + g) = rr;
        *reinterpret_cast<real2*>(qout + g) = qq;
        if (A.rhs_out) *reinterpret_cast<real2*>(A.rhs_out + g) = r;
      } else {
        *reinterpret_cast<real2*>(qout + g) = r;
      }
    }
  }
#undef GEO
}

}  // namespace REALNS
}  // namespace dgw
