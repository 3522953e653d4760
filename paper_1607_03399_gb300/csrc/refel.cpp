// Reference elements (see refel.hpp).  Written from the definitions:
// orthonormal Jacobi polynomials (Abramowitz & Stegun 22.7.1 recurrence and
// 22.8 derivative), collapsed-coordinate Proriol-Koornwinder-Dubiner bases,
// Gauss / Gauss-Lobatto points by Newton iteration, and Warburton's (2006)
// warp & blend node construction expressed in barycentric coordinates.
#include "refel.hpp"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace dgw {

const double kLSRK_A[5] = {0.0,
                           -567301805773.0 / 1357537059087.0,
                           -2404267990393.0 / 2016746695238.0,
                           -3550918686646.0 / 2091501179385.0,
                           -1275806237668.0 / 842570457699.0};
const double kLSRK_B[5] = {1432997174477.0 / 9575080441755.0,
                           5161836677717.0 / 13612068292357.0,
                           1720146321549.0 / 2090206949498.0,
                           3134564353537.0 / 4481467310338.0,
                           2277821191437.0 / 14882151754819.0};
const double kLSRK_C[5] = {0.0,
                           1432997174477.0 / 9575080441755.0,
                           2526269341429.0 / 6820363962896.0,
                           2006345519317.0 / 3224310063776.0,
                           2802321613138.0 / 2924317926251.0};

// ---------------------------------------------------------------- algebra
Mat matmul(const Mat& A, const Mat& B) {
  Mat C(A.r, B.c);
  for (int i = 0; i < A.r; ++i)
    for (int k = 0; k < A.c; ++k) {
      const double aik = A(i, k);
      for (int j = 0; j < B.c; ++j) C(i, j) += aik * B(k, j);
    }
  return C;
}

Mat transpose(const Mat& A) {
  Mat T(A.c, A.r);
  for (int i = 0; i < A.r; ++i)
    for (int j = 0; j < A.c; ++j) T(j, i) = A(i, j);
  return T;
}

bool invert(const Mat& A, Mat& Ainv) {
  const int n = A.r;
  Mat W = A;
  Ainv = Mat(n, n);
  for (int i = 0; i < n; ++i) Ainv(i, i) = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int i = col + 1; i < n; ++i)
      if (std::fabs(W(i, col)) > std::fabs(W(piv, col))) piv = i;
    if (std::fabs(W(piv, col)) < 1e-300) return false;
    if (piv != col)
      for (int j = 0; j < n; ++j) {
        std::swap(W(col, j), W(piv, j));
        std::swap(Ainv(col, j), Ainv(piv, j));
      }
    const double d = 1.0 / W(col, col);
    for (int j = 0; j < n; ++j) {
      W(col, j) *= d;
      Ainv(col, j) *= d;
    }
    for (int i = 0; i < n; ++i) {
      if (i == col) continue;
      const double f = W(i, col);
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        W(i, j) -= f * W(col, j);
        Ainv(i, j) -= f * Ainv(col, j);
      }
    }
  }
  return true;
}

// ------------------------------------------------------------ 1D polynomials
// Jacobi P_n^{(al,be)}(x), unnormalised (P_n(1) = binom(n+al, n)).
static double jacobi_raw(int n, double al, double be, double x) {
  if (n == 0) return 1.0;
  double pm = 1.0;
  double p = 0.5 * ((al + be + 2.0) * x + (al - be));
  for (int k = 1; k < n; ++k) {
    const double s = 2.0 * k + al + be;
    const double c1 = 2.0 * (k + 1) * (k + al + be + 1) * s;
    const double c2 = (s + 1) * ((s + 2) * s * x + al * al - be * be);
    const double c3 = 2.0 * (k + al) * (k + be) * (s + 2);
    const double pn = (c2 * p - c3 * pm) / c1;
    pm = p;
    p = pn;
  }
  return p;
}

// squared norm int_{-1}^{1} (1-x)^al (1+x)^be P_n^2
static double jacobi_norm2(int n, double al, double be) {
  const double lg = (al + be + 1.0) * std::log(2.0) - std::log(2.0 * n + al + be + 1.0) +
                    std::lgamma(n + al + 1.0) + std::lgamma(n + be + 1.0) -
                    std::lgamma(n + al + be + 1.0) - std::lgamma(n + 1.0);
  return std::exp(lg);
}

// orthonormal Jacobi polynomial and its derivative
static double jacobi(int n, double al, double be, double x) {
  return jacobi_raw(n, al, be, x) / std::sqrt(jacobi_norm2(n, al, be));
}
static double djacobi(int n, double al, double be, double x) {
  if (n == 0) return 0.0;
  return 0.5 * (n + al + be + 1.0) * jacobi_raw(n - 1, al + 1.0, be + 1.0, x) /
         std::sqrt(jacobi_norm2(n, al, be));
}

// Legendre P_n and P_n' by the three-term recurrence
static void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) {
    p = 1.0;
    dp = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    const double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1;
    p1 = p2;
    d0 = d1;
    d1 = d2;
  }
  p = p1;
  dp = d1;
}

static void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double z = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(q, z, p, dp);
      const double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre(q, z, p, dp);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static std::vector<double> gll_points(int N) {
  std::vector<double> x(N + 1);
  x[0] = -1.0;
  x[N] = 1.0;
  for (int k = 1; k < N; ++k) {
    double z = -std::cos(M_PI * k / N);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(N, z, p, dp);
      // P'' from the Legendre equation (1-z^2) P'' = 2 z P' - N(N+1) P
      const double d2p = (2.0 * z * dp - N * (N + 1.0) * p) / (1.0 - z * z);
      const double dz = dp / d2p;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[k] = z;
  }
  std::sort(x.begin(), x.end());
  return x;
}

// ------------------------------------------------------------ modal bases
// triangle: psi_ij = sqrt2 P_i(a) P_j^{(2i+1,0)}(b) (1-b)^i,
//   a = 2(1+r)/(1-s) - 1, b = s
static void tri_basis(int N, double r, double s, std::vector<double>& v,
                      std::vector<double>& vr, std::vector<double>& vs) {
  const double a = (std::fabs(1.0 - s) > 1e-14) ? 2.0 * (1.0 + r) / (1.0 - s) - 1.0 : -1.0;
  const double b = s;
  v.clear();
  vr.clear();
  vs.clear();
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j) {
      const double f = jacobi(i, 0, 0, a), df = djacobi(i, 0, 0, a);
      const double g = jacobi(j, 2.0 * i + 1, 0, b), dg = djacobi(j, 2.0 * i + 1, 0, b);
      const double ob = 1.0 - b;
      const double c = std::sqrt(2.0);
      v.push_back(c * f * g * std::pow(ob, i));
      double dr = 0.0, ds = 0.0;
      if (i >= 1) {
        dr = 2.0 * df * g * std::pow(ob, i - 1);
        ds = (1.0 + a) * df * g * std::pow(ob, i - 1) - i * f * g * std::pow(ob, i - 1);
      }
      ds += f * dg * std::pow(ob, i);
      vr.push_back(c * dr);
      vs.push_back(c * ds);
    }
}

// tet: psi_ijk = 2 sqrt2 P_i(a) P_j^{(2i+1,0)}(b) (1-b)^i P_k^{(2i+2j+2,0)}(c) (1-c)^{i+j}
static void tet_basis(int N, double r, double s, double t, std::vector<double>& v,
                      std::vector<double>& vr, std::vector<double>& vs, std::vector<double>& vt) {
  const double a = (std::fabs(s + t) > 1e-14) ? -2.0 * (1.0 + r) / (s + t) - 1.0 : -1.0;
  const double b = (std::fabs(1.0 - t) > 1e-14) ? 2.0 * (1.0 + s) / (1.0 - t) - 1.0 : -1.0;
  const double c = t;
  const double C = 2.0 * std::sqrt(2.0);
  v.clear();
  vr.clear();
  vs.clear();
  vt.clear();
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j)
      for (int k = 0; k <= N - i - j; ++k) {
        const double f = jacobi(i, 0, 0, a), df = djacobi(i, 0, 0, a);
        const double g = jacobi(j, 2.0 * i + 1, 0, b), dg = djacobi(j, 2.0 * i + 1, 0, b);
        const double h = jacobi(k, 2.0 * (i + j) + 2, 0, c), dh = djacobi(k, 2.0 * (i + j) + 2, 0, c);
        const double ob = 1.0 - b, oc = 1.0 - c;
        const int ij = i + j;
        v.push_back(C * f * g * std::pow(ob, i) * h * std::pow(oc, ij));
        // G_b' = d/db [g (1-b)^i], H_c' = d/dc [h (1-c)^{i+j}]
        double Gb = dg * std::pow(ob, i);
        if (i >= 1) Gb -= i * g * std::pow(ob, i - 1);
        double Hc = dh * std::pow(oc, ij);
        if (ij >= 1) Hc -= ij * h * std::pow(oc, ij - 1);
        double dr = 0.0, ds = 0.0, dt = 0.0;
        if (i >= 1) {
          const double base = df * g * h * std::pow(ob, i - 1) * std::pow(oc, ij - 1);
          dr = 4.0 * base;
          ds = 2.0 * (1.0 + a) * base;
          dt = 2.0 * (1.0 + a) * base;
        }
        if (ij >= 1) {
          ds += 2.0 * f * Gb * h * std::pow(oc, ij - 1);
          dt += (1.0 + b) * f * Gb * h * std::pow(oc, ij - 1);
        }
        dt += f * g * std::pow(ob, i) * Hc;
        vr.push_back(C * dr);
        vs.push_back(C * ds);
        vt.push_back(C * dt);
      }
}

// ------------------------------------------------------------ warp & blend
static const double kAlphaTet[15] = {0.0,    0.0,    0.0,    0.1002, 1.1332,
                                     1.5608, 1.3413, 1.2577, 1.1603, 1.10153,
                                     0.6080, 0.4523, 0.8856, 0.8717, 0.9655};

// Displacement interpolant on equispaced points mapping them to GLL points,
// divided by (1 - x^2).
static double warp_factor(int N, const std::vector<double>& gll, double x) {
  if (std::fabs(x) >= 1.0 - 1e-10) return 0.0;
  double w = 0.0;
  for (int i = 0; i <= N; ++i) {
    const double xi = -1.0 + 2.0 * i / N;
    double li = 1.0;
    for (int m = 0; m <= N; ++m) {
      if (m == i) continue;
      const double xm = -1.0 + 2.0 * m / N;
      li *= (x - xm) / (xi - xm);
    }
    w += (gll[i] - xi) * li;
  }
  return w / (1.0 - x * x);
}

// Barycentric displacement of a point from the 2D warp on the face spanned by
// vertices f[0..2] (indices into lam): every edge (a, b) with opposite vertex
// c pushes the point toward b by 4 lam_a lam_b warp(lam_b - lam_a)
// (1 + (alpha lam_c)^2) in units where an edge is 2 long.
static void face_warp(int N, const std::vector<double>& gll, double alpha, const double* lam,
                      const int* f, double* d) {
  for (int e = 0; e < 3; ++e) {
    const int a = f[e], b = f[(e + 1) % 3], c = f[(e + 2) % 3];
    const double w = 4.0 * lam[a] * lam[b] * warp_factor(N, gll, lam[b] - lam[a]) *
                     (1.0 + (alpha * lam[c]) * (alpha * lam[c]));
    d[b] += 0.5 * w;
    d[a] -= 0.5 * w;
  }
}

// ------------------------------------------------------------ build
RefElems build_reference(int N) {
  if (N < 1 || N > 8) throw std::runtime_error("order out of range");
  RefElems R;
  R.N = N;
  R.Nq = N + 1;
  R.Nt = (N + 1) * (N + 2) / 2;
  R.Npw = R.Nt * R.Nq;
  R.Npt = (N + 1) * (N + 2) * (N + 3) / 6;
  const int Nt = R.Nt, Nq = R.Nq, Npt = R.Npt;
  const double alpha = kAlphaTet[N - 1];
  R.gll = gll_points(N);

  // ---- line
  {
    Mat V(Nq, Nq), Vr(Nq, Nq), Vinv;
    for (int i = 0; i < Nq; ++i)
      for (int n = 0; n < Nq; ++n) {
        V(i, n) = jacobi(n, 0, 0, R.gll[i]);
        Vr(i, n) = djacobi(n, 0, 0, R.gll[i]);
      }
    invert(V, Vinv);
    R.line_Vinv = Vinv;
    Mat VVt = matmul(V, transpose(V));  // = (M^1D)^{-1}
    invert(VVt, R.M1);
    R.D1 = matmul(Vr, Vinv);
    R.ell0.resize(Nq);
    R.ellN.resize(Nq);
    for (int i = 0; i < Nq; ++i) {
      R.ell0[i] = VVt(i, 0);
      R.ellN[i] = VVt(i, N);
    }
    std::vector<double> xq, wq;
    gauss_legendre(N + 2, xq, wq);
    Mat Qa(Nq, Nq), Qb(Nq, Nq);
    for (size_t q = 0; q < xq.size(); ++q) {
      std::vector<double> P(Nq);
      for (int n = 0; n < Nq; ++n) P[n] = jacobi(n, 0, 0, xq[q]);
      for (int m = 0; m < Nq; ++m)
        for (int n = 0; n < Nq; ++n) {
          Qa(m, n) += wq[q] * 0.5 * (1.0 - xq[q]) * P[m] * P[n];
          Qb(m, n) += wq[q] * 0.5 * (1.0 + xq[q]) * P[m] * P[n];
        }
    }
    R.Mea = matmul(transpose(Vinv), matmul(Qa, Vinv));
    R.Meb = matmul(transpose(Vinv), matmul(Qb, Vinv));
  }

  // ---- triangle nodes (face distribution of the tet)
  std::vector<std::array<int, 2>> lat2;
  for (int b = 0; b <= N; ++b)
    for (int a = 0; a <= N - b; ++a) lat2.push_back({a, b});
  R.tri_r.resize(Nt);
  R.tri_s.resize(Nt);
  for (int n = 0; n < Nt; ++n) {
    double lam[3] = {double(N - lat2[n][0] - lat2[n][1]) / N, double(lat2[n][0]) / N,
                     double(lat2[n][1]) / N};
    double d[3] = {0, 0, 0};
    const int f[3] = {0, 1, 2};
    face_warp(N, R.gll, alpha, lam, f, d);
    const double l0 = lam[0] + d[0], l1 = lam[1] + d[1], l2 = lam[2] + d[2];
    R.tri_r[n] = -l0 + l1 - l2;
    R.tri_s[n] = -l0 - l1 + l2;
  }
  // ---- triangle operators
  {
    Mat V(Nt, Nt), Vr(Nt, Nt), Vs(Nt, Nt), Vinv;
    std::vector<double> v, vr, vs;
    for (int i = 0; i < Nt; ++i) {
      tri_basis(N, R.tri_r[i], R.tri_s[i], v, vr, vs);
      for (int m = 0; m < Nt; ++m) {
        V(i, m) = v[m];
        Vr(i, m) = vr[m];
        Vs(i, m) = vs[m];
      }
    }
    if (!invert(V, Vinv)) throw std::runtime_error("singular triangle Vandermonde");
    R.tri_Vinv = Vinv;
    R.Dr = matmul(Vr, Vinv);
    R.Ds = matmul(Vs, Vinv);
    Mat VVt = matmul(V, transpose(V));
    invert(VVt, R.Mt);
    // barycentric-weighted masses by collapsed Gauss quadrature
    std::vector<double> xg, wg;
    gauss_legendre(N + 2, xg, wg);
    Mat Q[3] = {Mat(Nt, Nt), Mat(Nt, Nt), Mat(Nt, Nt)};
    for (size_t ia = 0; ia < xg.size(); ++ia)
      for (size_t ib = 0; ib < xg.size(); ++ib) {
        const double A = xg[ia], B = xg[ib];
        const double r = 0.5 * (1 + A) * (1 - B) - 1.0, s = B;
        const double w = wg[ia] * wg[ib] * 0.5 * (1 - B);
        const double lam[3] = {-0.5 * (r + s), 0.5 * (1 + r), 0.5 * (1 + s)};
        tri_basis(N, r, s, v, vr, vs);
        for (int k = 0; k < 3; ++k)
          for (int m = 0; m < Nt; ++m)
            for (int n = 0; n < Nt; ++n) Q[k](m, n) += w * lam[k] * v[m] * v[n];
      }
    for (int k = 0; k < 3; ++k) R.Ma[k] = matmul(transpose(Vinv), matmul(Q[k], Vinv));
  }
  // ---- triangle edges: nodes ordered from the edge's first vertex to its second
  R.edge_nodes.assign(3, std::vector<int>(Nq));
  for (int m = 0; m <= N; ++m) {
    R.edge_nodes[0][m] = tri_index(N, m, 0);      // (v0 -> v1): b = 0, a = m
    R.edge_nodes[1][m] = tri_index(N, N - m, m);  // (v1 -> v2): a + b = N
    R.edge_nodes[2][m] = tri_index(N, 0, N - m);  // (v2 -> v0): a = 0
  }
  // ---- wedge faces
  R.wedge_face_nodes.assign(5, {});
  for (int i = 0; i < Nt; ++i) {
    R.wedge_face_nodes[0].push_back(i);
    R.wedge_face_nodes[1].push_back(N * Nt + i);
  }
  for (int e = 0; e < 3; ++e)
    for (int j = 0; j <= N; ++j)
      for (int m = 0; m <= N; ++m) R.wedge_face_nodes[2 + e].push_back(j * Nt + R.edge_nodes[e][m]);
  // ---- triangle face permutations
  R.tri_perm.assign(9, {});
  for (int p0 = 0; p0 < 3; ++p0)
    for (int p1 = 0; p1 < 3; ++p1) {
      if (p1 == p0) continue;
      const int pos[3] = {p0, p1, 3 - p0 - p1};
      std::vector<int>& P = R.tri_perm[p0 * 3 + p1];
      P.resize(Nt);
      for (int k = 0; k < Nt; ++k) {
        const int l[3] = {N - lat2[k][0] - lat2[k][1], lat2[k][0], lat2[k][1]};
        P[k] = tri_index(N, l[pos[1]], l[pos[2]]);
      }
    }

  // ---- tet nodes
  std::vector<std::array<int, 3>> lat3;
  for (int c = 0; c <= N; ++c)
    for (int b = 0; b <= N - c; ++b)
      for (int a = 0; a <= N - b - c; ++a) lat3.push_back({a, b, c});
  R.tet_r.resize(Npt);
  R.tet_s.resize(Npt);
  R.tet_t.resize(Npt);
  // faces as (opposite vertex, face vertices)
  const int fopp[4] = {3, 2, 0, 1};
  const int fvert[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};
  for (int n = 0; n < Npt; ++n) {
    const int li[4] = {N - lat3[n][0] - lat3[n][1] - lat3[n][2], lat3[n][0], lat3[n][1], lat3[n][2]};
    double lam[4];
    for (int k = 0; k < 4; ++k) lam[k] = double(li[k]) / N;
    int nzero = 0;
    for (int k = 0; k < 4; ++k) nzero += (li[k] == 0);
    double shift[4] = {0, 0, 0, 0};
    if (nzero >= 2) {
      // on an edge (or a vertex): the 1D warp of any face containing it
      for (int f = 0; f < 4; ++f)
        if (li[fopp[f]] == 0) {
          face_warp(N, R.gll, alpha, lam, fvert[f], shift);
          break;
        }
    } else {
      for (int f = 0; f < 4; ++f) {
        double d[4] = {0, 0, 0, 0};
        face_warp(N, R.gll, alpha, lam, fvert[f], d);
        const double La = lam[fopp[f]];
        const double l0 = lam[fvert[f][0]], l1 = lam[fvert[f][1]], l2 = lam[fvert[f][2]];
        double blend = l0 * l1 * l2;
        const double den = (l0 + 0.5 * La) * (l1 + 0.5 * La) * (l2 + 0.5 * La);
        if (den > 1e-10) blend = (1.0 + (alpha * La) * (alpha * La)) * blend / den;
        for (int k = 0; k < 4; ++k) shift[k] += blend * d[k];
      }
    }
    double L[4];
    for (int k = 0; k < 4; ++k) L[k] = lam[k] + shift[k];
    // vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1), (-1,-1,1)
    R.tet_r[n] = -L[0] + L[1] - L[2] - L[3];
    R.tet_s[n] = -L[0] - L[1] + L[2] - L[3];
    R.tet_t[n] = -L[0] - L[1] - L[2] + L[3];
  }
  R.tet_face_nodes.assign(4, {});
  for (int n = 0; n < Npt; ++n) {
    const int a = lat3[n][0], b = lat3[n][1], c = lat3[n][2];
    if (c == 0) R.tet_face_nodes[0].push_back(n);
    if (b == 0) R.tet_face_nodes[1].push_back(n);
    if (a + b + c == N) R.tet_face_nodes[2].push_back(n);
    if (a == 0) R.tet_face_nodes[3].push_back(n);
  }
  {
    Mat V(Npt, Npt), Vr(Npt, Npt), Vs(Npt, Npt), Vt(Npt, Npt), Vinv;
    std::vector<double> v, vr, vs, vt;
    for (int i = 0; i < Npt; ++i) {
      tet_basis(N, R.tet_r[i], R.tet_s[i], R.tet_t[i], v, vr, vs, vt);
      for (int m = 0; m < Npt; ++m) {
        V(i, m) = v[m];
        Vr(i, m) = vr[m];
        Vs(i, m) = vs[m];
        Vt(i, m) = vt[m];
      }
    }
    if (!invert(V, Vinv)) throw std::runtime_error("singular tet Vandermonde");
    R.tet_Vinv = Vinv;
    R.tDr = matmul(Vr, Vinv);
    R.tDs = matmul(Vs, Vinv);
    R.tDt = matmul(Vt, Vinv);
    Mat VVt = matmul(V, transpose(V));  // (M^tet)^{-1}
    invert(VVt, R.tM);
    R.tLIFT = Mat(Npt, 4 * Nt);
    for (int f = 0; f < 4; ++f)
      for (int i = 0; i < Npt; ++i)
        for (int k = 0; k < Nt; ++k) {
          double acc = 0.0;
          for (int l = 0; l < Nt; ++l) acc += VVt(i, R.tet_face_nodes[f][l]) * R.Mt(l, k);
          R.tLIFT(i, f * Nt + k) = acc;
        }
  }
  return R;
}

void line_lagrange(const RefElems& R, double t, double* out) {
  for (int j = 0; j < R.Nq; ++j) {
    double v = 0.0;
    for (int n = 0; n < R.Nq; ++n) v += jacobi(n, 0, 0, t) * R.line_Vinv(n, j);
    out[j] = v;
  }
}

void tri_lagrange(const RefElems& R, double r, double s, double* out) {
  std::vector<double> v, vr, vs;
  tri_basis(R.N, r, s, v, vr, vs);
  for (int i = 0; i < R.Nt; ++i) {
    double acc = 0.0;
    for (int m = 0; m < R.Nt; ++m) acc += v[m] * R.tri_Vinv(m, i);
    out[i] = acc;
  }
}

void tet_lagrange(const RefElems& R, double r, double s, double t, double* out) {
  std::vector<double> v, vr, vs, vt;
  tet_basis(R.N, r, s, t, v, vr, vs, vt);
  for (int i = 0; i < R.Npt; ++i) {
    double acc = 0.0;
    for (int m = 0; m < R.Npt; ++m) acc += v[m] * R.tet_Vinv(m, i);
    out[i] = acc;
  }
}

}  // namespace dgw
