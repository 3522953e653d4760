// Receiver sampling, adjoint source injection and the gradient kernel of the
// discrete adjoint (included by kernels.cuh once per precision and order,
// after the stage kernels whose helpers it uses).
#pragma once

namespace dgw {
namespace REALNS {

// ---------------------------------------------------------------------------
// receivers and the adjoint (gradient with respect to kappa and rho)
// ---------------------------------------------------------------------------
// packed index of field slot 0 (pressure) of node n of the element (type, e)
template <int N>
__device__ __forceinline__ int64_t pidx(const DevMesh<real>& M, int type, int e, int n) {
  return type == 6 ? widx<N>(e >> 5, n, e & 31) : tidx<N>(M.tet_off, e >> 5, n, e & 31);
}

// out[shot][r] = sum_n l_r(n) p(n) in the receiver's element of that shot
template <int N>
__global__ void k_sample(const DevMesh<real> M, const real* __restrict__ q, real* __restrict__ out, int nshots) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nshots * M.nrec) return;
  const int shot = idx / M.nrec, r = idx - shot * M.nrec;
  const RecDev rd = M.rec[r];
  const int e = int(shot_vid(shot, rd.elem, rd.type == 6 ? M.Kw1 : M.Kt1, M.shot_group));
  const int np = rd.type == 6 ? npw_of(N) : npt_of(N);
  real acc = 0;
  for (int n = 0; n < np; ++n) acc += M.rec_l[rd.loff + n] * q[pidx<N>(M, rd.type, e, n)];
  out[idx] = acc;
}

// Adjoint load of the misfit residuals (in the variables mu = P W^{-1} lambda):
// mu_Q,p += kappa (M^k)^{-1} sum_r resid_r l(x_r) on each receiver element, and
// the next stage input x += b5 times the same.  One thread per (shot, element
// group), receivers of a group in list order: deterministic.
template <int N>
__global__ void k_inject(const DevMesh<real> M, real* __restrict__ muq, real* __restrict__ x,
                         const real* __restrict__ resid, int nshots, real b5) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nshots * M.nrgrp) return;
  const int shot = idx / M.nrgrp, gi = idx - shot * M.nrgrp;
  const RecGroup g = M.rgrp[gi];
  const int e = int(shot_vid(shot, g.elem, g.type == 6 ? M.Kw1 : M.Kt1, M.shot_group));
  const real kappa = g.type == 6 ? M.w_mat[e] : M.t_mat[e];
  const int np = g.type == 6 ? npw_of(N) : npt_of(N);
  for (int n = 0; n < np; ++n) {
    real acc = 0;
    for (int i = g.r0; i < g.r0 + g.nr; ++i) {
      const int r = M.rperm[i];
      acc += resid[shot * M.nrec + r] * M.rec_g[M.rec[r].loff + n];
    }
    const int64_t i = pidx<N>(M, g.type, e, n);
    muq[i] += kappa * acc;
    x[i] += b5 * kappa * acc;
  }
}

// Per wedge and Runge-Kutta stage, with x = mu_K (adjoint stage variable,
// lambda_K = W P mu_K), q = the forward stage input Q and r = A Q + f its
// right-hand side:
//   d/dkappa_k: mu_p^T M^k r_p / kappa^2 + dz/dkappa G,  d/drho_k: mu_u^T M^k r_u + dz/drho G,
// with z = rho c = sqrt(kappa rho) and G the derivative of the upwind penalty
// in z summed over the element's faces: interior faces (tau_p = 2/(z- + z+),
// tau_u = (z- + z+)/2) give tau_p^2/4 int [p][mu_p] + 1/4 int [u_n][mu_un],
// rigid walls int mu_un u_n, Dirichlet walls int mu_p p / z^2; central fluxes
// have no penalty.  M^k = M^{tri,k} (x) M^1D (Section 4.2); the face masses are
// J_f M^tri (triangles) and M~_e (x) M^1D (quadrilaterals).  A CTA takes a
// 32-wedge block with N+1 warps (slabs of x and q in shared memory): warp j
// forms the element terms of slice j and the face terms of the faces it is
// given (grad_tri_warp and quadrilateral face e on warp e mod (N+1)); the
// warps' partial element sums are reduced in a fixed order and added, times
// dt, in double; the face terms go to per-face sums (dz/dkappa and dz/drho
// applied when the gradient is read).  The right-hand side is read from
// global memory, one slice per warp (staging it as a third slab measured
// slower at N = 3: fewer CTAs per SM).
// Shared memory: x slab, q slab, geometry, [warp][3][32] partial sums, the
// copy barrier and the failure flag.
template <int N>
__host__ __device__ constexpr int grad_smem_bytes() {
  constexpr int Nt = nt_of(N), Nq = N + 1, Np = Nt * Nq;
  return int(sizeof(real)) * (2 * 4 * Np * kB + G_COUNT * kB) + 8 * 3 * Nq * kB + 16;
}

// the warp that owns triangle face fb (0 bottom, 1 top) in the gradient
// kernel: the warps left over after the three quadrilateral faces
__host__ __device__ constexpr int grad_tri_warp(int N, int fb) {
  return N >= 4 ? 3 + fb : (N == 3 ? 3 : (N == 2 ? fb : 1));
}

// TETS: the mesh has tets, so a triangle face may neighbour one (wedge-only
// meshes take the instantiation without that branch)
template <int N, bool TETS>
__global__ void __launch_bounds__(32 * (N + 1), (sizeof(real) == 4) ? (N <= 3 ? 4 : 2) : (N <= 3 ? 2 : 1))
    k_wedge_grad(const DevMesh<real> M, const real* __restrict__ X,
                                                             const real* __restrict__ Q, const real* __restrict__ R,
                                                             double dt, int flux, int bc, double* __restrict__ gk,
                                                             double* __restrict__ gr, double* __restrict__ gz) {
  constexpr int Nt = nt_of(N), Nq = N + 1, Np = Nt * Nq;
  const AllOps<N, real>& O = OPS<N>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  real* sX = reinterpret_cast<real*>(smem_raw);
  real* sQ = sX + 4 * Np * kB;
  real* sG = sQ + 4 * Np * kB;
  double* red = reinterpret_cast<double*>(sG + G_COUNT * kB);  // [warp][3][32]
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + 3 * Nq * kB);  // slabs and coordinates
  int* failed = reinterpret_cast<int*>(bar + 1);
  const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;
  const int blk = blockIdx.x, e = blk * kB + lane;
  const int Kp = M.Kw_pad;
  constexpr uint32_t slab_bytes = uint32_t(4 * Np * kB * sizeof(real)), xyz_bytes = uint32_t(12 * kB * sizeof(real));
  if (threadIdx.x == 0) {
    *failed = 0;
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_expect_tx(bar, 2 * slab_bytes + xyz_bytes);
    bulk_g2s(sX, X + int64_t(blk) * 4 * Np * kB, slab_bytes, bar);
    bulk_g2s(sQ, Q + int64_t(blk) * 4 * Np * kB, slab_bytes, bar);
    bulk_g2s(sG, M.w_xyz + int64_t(blk) * 12 * kB, xyz_bytes, bar);
  }
  // this slice of the right-hand side, the material and the face neighbours
  // (ids, codes, impedances), in flight while the slabs arrive
  Q4 rj[Nt];
#pragma unroll
  for (int i = 0; i < Nt; ++i) rj[i] = ld4(R, widx<N>(blk, j * Nt + i, lane));
  const real kappa = M.w_mat[0 * Kp + e], zM = M.w_mat[2 * Kp + e];
  int nbf[5], cdf[5];
  real zPf[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    nbf[f] = M.w_nbr[f * Kp + e];
    cdf[f] = M.w_code[f * Kp + e];
  }
#pragma unroll
  for (int f = 0; f < 5; ++f)
    zPf[f] = nbf[f] < 0 ? zM
                        : ((TETS && f < 2 && (cdf[f] & kCodeTet)) ? M.t_mat[2 * M.Kt_pad + nbf[f]]
                                                                   : M.w_mat[2 * Kp + nbf[f]]);
  __syncthreads();
  if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar, 0)) && lane == 0) atomicOr(failed, 1);
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(failed)) {
    // the copies never completed: report, let them drain, every warp leaves
    if (threadIdx.x == 0) {
      atomicOr(M.err, kErrTimeout);
      mbar_wait_bounded(bar, 0);
    }
    return;
  }
  if (j == 0) wedge_geometry(sG, lane);
  __syncthreads();
#define GEO(item) sG[(item) * kB + lane]
  const real J0 = GEO(G_J0), J1 = GEO(G_J1), J2 = GEO(G_J2);

  // element terms: mu^T (M^tri (x) M^1D) r = sum_j' (sum_j M1[j][j'] mu[j])^T M^tri r[j'];
  // warp j takes the term of r's slice j (its own, loaded once from global
  // memory) and the M1-weighted sum of the mu slices from the shared slab
  // (packed pairs: the mu sums by field pairs (p, u_x), (u_y, u_z); the
  // entries of M^{tri,k} two rows at a time from the output-pair tables)
  real t1k = 0, t1r = 0;
  {
    real2 b01[Nt], b23[Nt];
#pragma unroll
    for (int l = 0; l < Nt; ++l) b01[l] = b23[l] = dup2(real(0));
#pragma unroll
    for (int jp = 0; jp < Nq; ++jp) {
      const real2 m1 = dup2(O.w.M1[jp * Nq + j]);
#pragma unroll
      for (int l = 0; l < Nt; ++l) {
        const Q4 v = lds4(sX, jp * Nt + l, lane);
        b01[l] = fma2(m1, mk2(v.p, v.u), b01[l]);
        b23[l] = fma2(m1, mk2(v.v, v.w), b23[l]);
      }
    }
    const real2 J0d = dup2(J0), J1d = dup2(J1), J2d = dup2(J2);
    constexpr int NH = (Nt + 1) / 2;
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      // rows i0 = 2h and i1 = 2h + 1 (an odd last row pairs with a zero row)
      real2 c01a = dup2(real(0)), c23a = dup2(real(0)), c01b = dup2(real(0)), c23b = dup2(real(0));
#pragma unroll
      for (int l = 0; l < Nt; ++l) {
        const real2 mt = fma2(cpair(O.w.MaP[0], Nt, h, l), J0d,
                              fma2(cpair(O.w.MaP[1], Nt, h, l), J1d, mul2(cpair(O.w.MaP[2], Nt, h, l), J2d)));
        const real2 ma = dup2(mt.x), mb = dup2(mt.y);
        c01a = fma2(ma, b01[l], c01a);
        c23a = fma2(ma, b23[l], c23a);
        c01b = fma2(mb, b01[l], c01b);
        c23b = fma2(mb, b23[l], c23b);
      }
      const Q4 ra = rj[2 * h];
      t1k += ra.p * c01a.x;
      t1r += ra.u * c01a.y + ra.v * c23a.x + ra.w * c23a.y;
      if (2 * h + 1 < Nt) {
        const Q4 rb = rj[2 * h + 1];
        t1k += rb.p * c01b.x;
        t1r += rb.u * c01b.y + rb.v * c23b.x + rb.w * c23b.y;
      }
    }
  }
  t1k /= kappa * kappa;

  // face terms: derivative of the upwind penalty in z.  Each face is one
  // warp's task (quadrilateral face e on warp e mod (N+1), the triangle faces
  // on the last warps): the warp forms the jumps of the whole face and its
  // face-mass integrals, with no exchange between warps.  The penalty term of
  // a face is symmetric in its two elements (tau_p, tau_u and the jump
  // products do not change with the side), so a face between two wedges is
  // evaluated once, by the lower-numbered wedge, which adds dt times it to
  // the face sums gz[face][element] of both; boundary faces and faces towards
  // a tet belong to the wedge.  Each face sum has one writer per launch.
  auto add_face = [&](int f, int nbr, int nf, real val) {
    const double v = dt * double(val);
    gz[int64_t(f) * Kp + e] += v;
    if (nbr >= 0) gz[int64_t(nf) * Kp + nbr] += v;
  };
  if (flux == 0) {
    // a neighbour's node value, from global memory also when the neighbour is
    // in this block (a uniform load stream measured faster than choosing the
    // shared slab per lane)
    auto nbv = [&](const real* glob, int nbr, int node) { return ld4(glob, widx<N>(nbr >> 5, node, nbr & 31)); };
    auto penalty = [&](int nbr, real zP, real Ip, real Iu) {
      if (nbr >= 0) {
        const real tp = real(2) / (zM + zP);
        return real(0.25) * tp * tp * Ip + real(0.25) * Iu;
      }
      return bc == 0 ? Ip / (zM * zM) : Iu;
    };
    // quadrilateral face ed (face mass M~_e (x) M^1D over slice jj, edge node m)
#pragma unroll 1
    for (int ed = j; ed < 3; ed += Nq) {
      const int nbr = ed == 0 ? nbf[2] : (ed == 1 ? nbf[3] : nbf[4]);
      const int code = ed == 0 ? cdf[2] : (ed == 1 ? cdf[3] : cdf[4]);
      const real zP = ed == 0 ? zPf[2] : (ed == 1 ? zPf[3] : zPf[4]);
      if (nbr >= 0 && nbr < e) continue;  // the neighbour's task
      const real nx = GEO(G_QNX0 + ed), ny = GEO(G_QNY0 + ed);
      const real ca = GEO(G_QCA0 + ed), cbq = GEO(G_QCB0 + ed);
      const int ep = nbr < 0 ? ed : code >> 1, rev = nbr < 0 ? 0 : code & 1;
      real b[Nq][Nq], d[Nq][Nq];  // [mu_p], [mu_un] (boundary: own values)
#pragma unroll
      for (int jj = 0; jj < Nq; ++jj)
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          const Q4 xo = lds4(sX, jj * Nt + edge_node(N, ed, m), lane);
          if (nbr < 0) {
            b[jj][m] = xo.p;
            d[jj][m] = nx * xo.u + ny * xo.v;
          } else {
            const Q4 xn = nbv(X, nbr, jj * Nt + O.tab.edge[ep][rev ? N - m : m]);
            b[jj][m] = xn.p - xo.p;
            d[jj][m] = nx * (xn.u - xo.u) + ny * (xn.v - xo.v);
          }
        }
      // (M^1D (x) M~_e) [mu]: along the slices, then along the edge
      real w[Nq][Nq];
#pragma unroll
      for (int m = 0; m < Nq; ++m)
#pragma unroll
        for (int mp = 0; mp < Nq; ++mp) w[m][mp] = ca * O.w.Mea[m * Nq + mp] + cbq * O.w.Meb[m * Nq + mp];
      real Bb[Nq][Nq], Bd[Nq][Nq];
#pragma unroll
      for (int jj = 0; jj < Nq; ++jj) {
        real tb[Nq], td[Nq];
#pragma unroll
        for (int mp = 0; mp < Nq; ++mp) {
          real sb = 0, sd = 0;
#pragma unroll
          for (int jp = 0; jp < Nq; ++jp) {
            sb += O.w.M1[jj * Nq + jp] * b[jp][mp];
            sd += O.w.M1[jj * Nq + jp] * d[jp][mp];
          }
          tb[mp] = sb;
          td[mp] = sd;
        }
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          real sb = 0, sd = 0;
#pragma unroll
          for (int mp = 0; mp < Nq; ++mp) {
            sb += w[m][mp] * tb[mp];
            sd += w[m][mp] * td[mp];
          }
          Bb[jj][m] = sb;
          Bd[jj][m] = sd;
        }
      }
      // [q] against it, node by node
      real Ip = 0, Iu = 0;
#pragma unroll
      for (int jj = 0; jj < Nq; ++jj)
#pragma unroll
        for (int m = 0; m < Nq; ++m) {
          const Q4 qo = lds4(sQ, jj * Nt + edge_node(N, ed, m), lane);
          real a, c;  // [p], [u_n] (boundary: own values)
          if (nbr < 0) {
            a = qo.p;
            c = nx * qo.u + ny * qo.v;
          } else {
            const Q4 qn = nbv(Q, nbr, jj * Nt + O.tab.edge[ep][rev ? N - m : m]);
            a = qn.p - qo.p;
            c = nx * (qn.u - qo.u) + ny * (qn.v - qo.v);
          }
          Ip += a * Bb[jj][m];
          Iu += c * Bd[jj][m];
        }
      add_face(2 + ed, nbr, 2 + ep, penalty(nbr, zP, Ip, Iu));
    }
    // triangle face fb (bottom, top; face mass J_f M^tri)
#pragma unroll 1
    for (int fb = 0; fb < 2; ++fb) {
      if (j != grad_tri_warp(N, fb)) continue;
      const int nbr = fb ? nbf[1] : nbf[0], code = fb ? cdf[1] : cdf[0];
      const real n0 = GEO(fb ? G_NT0 : G_NB0), n1 = GEO(fb ? G_NT1 : G_NB1), n2 = GEO(fb ? G_NT2 : G_NB2);
      const real Jf = GEO(fb ? G_JFT : G_JFB);
      const real zP = fb ? zPf[1] : zPf[0];
      // the neighbour across a triangle face: a wedge (its bottom or top slice) or,
      // at the wedge/tet interface, a tet (one of its faces)
      const bool ntet = TETS && nbr >= 0 && (code & kCodeTet) != 0;
      if (nbr >= 0 && !ntet && nbr < e) continue;  // the neighbour's task
      const int own0 = fb ? N * Nt : 0, nf = (code >> 4) & 3;
      auto nbt = [&](const real* glob, int k) {
        const int nk = O.tab.tri_perm[code & 15][k];
        return ntet ? ld4(glob, tidx<N>(M.tet_off, nbr >> 5, O.tab.tet_face[nf][nk], nbr & 31))
                    : ld4(glob, widx<N>(nbr >> 5, (nf ? N * Nt : 0) + nk, nbr & 31));
      };
      real a[Nt], b[Nt], c[Nt], d[Nt];  // [p], [mu_p], [u_n], [mu_un] (boundary: own values)
#pragma unroll
      for (int k = 0; k < Nt; ++k) {
        const Q4 qo = lds4(sQ, own0 + k, lane), xo = lds4(sX, own0 + k, lane);
        if (nbr < 0) {
          a[k] = qo.p;
          b[k] = xo.p;
          c[k] = n0 * qo.u + n1 * qo.v + n2 * qo.w;
          d[k] = n0 * xo.u + n1 * xo.v + n2 * xo.w;
        } else {
          const Q4 qn = nbt(Q, k), xn = nbt(X, k);
          a[k] = qn.p - qo.p;
          b[k] = xn.p - xo.p;
          c[k] = n0 * (qn.u - qo.u) + n1 * (qn.v - qo.v) + n2 * (qn.w - qo.w);
          d[k] = n0 * (xn.u - xo.u) + n1 * (xn.v - xo.v) + n2 * (xn.w - xo.w);
        }
      }
      real Ip = 0, Iu = 0;
#pragma unroll
      for (int k = 0; k < Nt; ++k) {
        real sp = 0, su = 0;
#pragma unroll
        for (int kk = 0; kk < Nt; ++kk) {
          sp += O.w.M[k * Nt + kk] * b[kk];
          su += O.w.M[k * Nt + kk] * d[kk];
        }
        Ip += a[k] * sp;
        Iu += c[k] * su;
      }
      add_face(fb, ntet ? -1 : nbr, nf, penalty(nbr, zP, Ip * Jf, Iu * Jf));
    }
  }
  // reduce the warps' partial sums in a fixed order
  red[(j * 3 + 0) * kB + lane] = double(t1k);
  red[(j * 3 + 1) * kB + lane] = double(t1r);
  __syncthreads();
  if (j == 0 && e < M.Kw) {
    double sk = 0.0, sr = 0.0;
    for (int jj = 0; jj < Nq; ++jj) {
      sk += red[(jj * 3 + 0) * kB + lane];
      sr += red[(jj * 3 + 1) * kB + lane];
    }
    gk[e] += dt * sk;
    gr[e] += dt * sr;
  }
#undef GEO
}

// The same gradient terms on the tets (affine: M^k = J M^tet with the reference
// tet mass, face mass J_f M^tri): per tet, J mu_p^T M^tet r_p / kappa^2 + dz/dkappa G
// and J mu_u^T M^tet r_u + dz/drho G, G the penalty derivative summed over the four
// faces, whose neighbours are tets or, across the interface, wedges.  CTA = a
// 32-tet block x 4 warps; the block's mu and r slabs in shared memory; warp w
// takes face w and element-term rows [w C, w C + C); the partial sums are
// reduced in a fixed order and added, times dt, in double.
template <int N>
__host__ __device__ constexpr int tgrad_smem_bytes() {
  return int(sizeof(real)) * 2 * 4 * npt_of(N) * kB + 8 * 3 * 4 * kB;
}

template <int N>
__global__ void __launch_bounds__(128) k_tet_grad(const DevMesh<real> M, const real* __restrict__ X,
                                                  const real* __restrict__ Q, const real* __restrict__ R, double dt,
                                                  int flux, int bc, double* __restrict__ gk, double* __restrict__ gr) {
  constexpr int Np = npt_of(N), Nt = nt_of(N), C = (Np + 3) / 4;
  const AllOps<N, real>& O = OPS<N>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  real* sX = reinterpret_cast<real*>(smem_raw);              // [Np][32][4]
  real* sR = sX + 4 * Np * kB;                                // [Np][32][4]
  double* red = reinterpret_cast<double*>(sR + 4 * Np * kB);  // [warp][3][32]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int blk = blockIdx.x, e = blk * kB + lane;
  const int Kp = M.Kt_pad;
  const int64_t base = tidx<N>(M.tet_off, blk, 0, 0);  // the block's [Np][32][4] records
  for (int i = threadIdx.x; i < Np * kB; i += blockDim.x) {
    const Q4 x = ld4(X, base + int64_t(i) * 4), r = ld4(R, base + int64_t(i) * 4);
    sX[i * 4 + 0] = x.p;
    sX[i * 4 + 1] = x.u;
    sX[i * 4 + 2] = x.v;
    sX[i * 4 + 3] = x.w;
    sR[i * 4 + 0] = r.p;
    sR[i * 4 + 1] = r.u;
    sR[i * 4 + 2] = r.v;
    sR[i * 4 + 3] = r.w;
  }
  const real kappa = M.t_mat[0 * Kp + e], irho = M.t_mat[1 * Kp + e], zM = M.t_mat[2 * Kp + e];
  // affine geometry (bi-unit reference tet): J, and face w's outward normal and J_f
  real J, n0, n1, n2, Jf;
  {
    real Xv[4][3];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int d = 0; d < 3; ++d) Xv[v][d] = M.t_xyz[(int64_t(blk) * 12 + v * 3 + d) * kB + lane];
    real G[3][3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int m = 0; m < 3; ++m) G[d][m] = real(0.5) * (Xv[m + 1][d] - Xv[0][d]);
    J = G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) - G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
        G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
    constexpr int fv[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};
    constexpr int fo[4] = {3, 2, 0, 1};
    const int a0 = w == 0 ? fv[0][0] : w == 1 ? fv[1][0] : w == 2 ? fv[2][0] : fv[3][0];
    const int a1 = w == 0 ? fv[0][1] : w == 1 ? fv[1][1] : w == 2 ? fv[2][1] : fv[3][1];
    const int a2 = w == 0 ? fv[0][2] : w == 1 ? fv[1][2] : w == 2 ? fv[2][2] : fv[3][2];
    const int ao = fo[0] * (w == 0) + fo[1] * (w == 1) + fo[2] * (w == 2) + fo[3] * (w == 3);
    real P[4][3];  // the face's vertices and the opposite one, selected without dynamic indexing
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      real v0 = 0, v1 = 0, v2 = 0, vo = 0;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        v0 = a0 == v ? Xv[v][d] : v0;
        v1 = a1 == v ? Xv[v][d] : v1;
        v2 = a2 == v ? Xv[v][d] : v2;
        vo = ao == v ? Xv[v][d] : vo;
      }
      P[0][d] = v0;
      P[1][d] = v1;
      P[2][d] = v2;
      P[3][d] = vo;
    }
    const real ax = P[1][0] - P[0][0], ay = P[1][1] - P[0][1], az = P[1][2] - P[0][2];
    const real bx = P[2][0] - P[0][0], by = P[2][1] - P[0][1], bz = P[2][2] - P[0][2];
    const real cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
    const real cc = cx * cx + cy * cy + cz * cz, ic = rsqrt_r(cc);
    const real ox = P[3][0] - P[0][0], oy = P[3][1] - P[0][1], oz = P[3][2] - P[0][2];
    const real sgn = (cx * ox + cy * oy + cz * oz > 0) ? real(-1) : real(1);  // away from the opposite vertex
    n0 = sgn * cx * ic;
    n1 = sgn * cy * ic;
    n2 = sgn * cz * ic;
    Jf = real(0.25) * cc * ic;
  }
  __syncthreads();

  // element terms, rows [w C, w C + C): mu_i . (M^tet r)_i
  real t1k = 0, t1r = 0;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    const int i = w * C + c;
    if (i < Np) {
      real c0 = 0, c1 = 0, c2 = 0, c3 = 0;
      for (int l = 0; l < Np; ++l) {
        const real m = M.tet_mass[i * Np + l];
        const Q4 r = lds4(sR, l, lane);
        c0 += m * r.p;
        c1 += m * r.u;
        c2 += m * r.v;
        c3 += m * r.w;
      }
      const Q4 x = lds4(sX, i, lane);
      t1k += x.p * c0;
      t1r += x.u * c1 + x.v * c2 + x.w * c3;
    }
  }
  t1k *= J / (kappa * kappa);
  t1r *= J;

  // penalty terms of face w
  real gz = 0;
  if (flux == 0) {
    const int f = w;
    const int nbr = M.t_nbr[f * Kp + e], code = M.t_code[f * Kp + e];
    const bool bnd = nbr < 0, ntet = !bnd && (code & kCodeTet) != 0;
    const real zP = bnd ? zM : (ntet ? M.t_mat[2 * Kp + nbr] : M.w_mat[2 * M.Kw_pad + nbr]);
    const int nfc = (code >> 4) & 3, perm = code & 15;
    real a[Nt], b[Nt], cq[Nt], d[Nt];  // [p], [mu_p], [u_n], [mu_un] (boundary: own values)
#pragma unroll
    for (int k = 0; k < Nt; ++k) {
      const int own = O.tab.tet_face[f][k];
      const Q4 qo = ld4(Q, base + (int64_t(own) * kB + lane) * 4), xo = lds4(sX, own, lane);
      if (bnd) {
        a[k] = qo.p;
        b[k] = xo.p;
        cq[k] = n0 * qo.u + n1 * qo.v + n2 * qo.w;
        d[k] = n0 * xo.u + n1 * xo.v + n2 * xo.w;
      } else {
        const int nk = O.tab.tri_perm[perm][k];
        const int node = ntet ? O.tab.tet_face[nfc][nk] : (nfc ? N * Nt : 0) + nk;
        const int64_t g = ntet ? tidx<N>(M.tet_off, nbr >> 5, node, nbr & 31) : widx<N>(nbr >> 5, node, nbr & 31);
        const Q4 qn = ld4(Q, g), xn = ld4(X, g);
        a[k] = qn.p - qo.p;
        b[k] = xn.p - xo.p;
        cq[k] = n0 * (qn.u - qo.u) + n1 * (qn.v - qo.v) + n2 * (qn.w - qo.w);
        d[k] = n0 * (xn.u - xo.u) + n1 * (xn.v - xo.v) + n2 * (xn.w - xo.w);
      }
    }
    real Ip = 0, Iu = 0;
#pragma unroll
    for (int k = 0; k < Nt; ++k) {
      real sp = 0, su = 0;
#pragma unroll
      for (int kk = 0; kk < Nt; ++kk) {
        sp += O.w.M[k * Nt + kk] * b[kk];
        su += O.w.M[k * Nt + kk] * d[kk];
      }
      Ip += a[k] * sp;
      Iu += cq[k] * su;
    }
    Ip *= Jf;
    Iu *= Jf;
    if (!bnd) {
      const real tp = real(2) / (zM + zP);
      gz = real(0.25) * tp * tp * Ip + real(0.25) * Iu;
    } else {
      gz = bc == 0 ? Ip / (zM * zM) : Iu;
    }
  }
  // reduce the warps' partial sums in a fixed order
  red[(w * 3 + 0) * kB + lane] = double(t1k);
  red[(w * 3 + 1) * kB + lane] = double(t1r);
  red[(w * 3 + 2) * kB + lane] = double(gz);
  __syncthreads();
  if (w == 0 && e < M.Kt) {
    double sk = 0.0, sr = 0.0, sz = 0.0;
    for (int ww = 0; ww < 4; ++ww) {
      sk += red[(ww * 3 + 0) * kB + lane];
      sr += red[(ww * 3 + 1) * kB + lane];
      sz += red[(ww * 3 + 2) * kB + lane];
    }
    const double rho = 1.0 / double(irho);
    gk[e] += dt * (sk + sz * double(zM) / (2.0 * double(kappa)));
    gr[e] += dt * (sr + sz * double(zM) / (2.0 * rho));
  }
}

}  // namespace REALNS
}  // namespace dgw
