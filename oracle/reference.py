"""Reference elements for the oracle (Section 3 and 3.1 of the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Reference domains (bi-unit, Section 3):
  line      [-1, 1]
  triangle  T = {r >= -1, s >= -1, r + s <= 0}, vertices (-1,-1), (1,-1), (-1,1)
  tet       {r, s, t >= -1, r + s + t <= -1}, vertices (-1,-1,-1), (1,-1,-1),
            (-1,1,-1), (-1,-1,1)
  wedge     T x [-1, 1]; node (i, j) = triangle node i, line node j, stored
            slice-major: n = j * Nt + i.

Nodes (Section 3.1): Gauss-Legendre-Lobatto on the line; Warp & Blend points
(Warburton 2006) on the tet, and on the triangle the tet's face distribution
(the wedge takes "nodes on the triangular face of the tetrahedron"), i.e. the
2D warp & blend with the tetrahedron's blend parameter alpha(N).

All matrices are built from their definitions: Lagrange basis functions are
evaluated through a total-degree Legendre-product Vandermonde, mass matrices
by Gauss (collapsed Duffy) quadrature exact for the integrand's degree, and
derivative matrices by differentiating the interpolant.

Canonical node orders (shared convention with the library's header):
  triangle: for b = 0..N, for a = 0..N-b   (lambda_2 = a/N, lambda_3 = b/N)
  tet:      for c = 0..N, for b = 0..N-c, for a = 0..N-b-c
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
from numpy.polynomial import legendre as npleg

# Warburton (2006) optimised blend parameters for the tetrahedron, N = 1..15.
ALPHA_TET = (0.0, 0.0, 0.0, 0.1002, 1.1332, 1.5608, 1.3413, 1.2577, 1.1603,
             1.10153, 0.6080, 0.4523, 0.8856, 0.8717, 0.9655)


def alpha_tet(N: int) -> float:
    return ALPHA_TET[N - 1] if N <= len(ALPHA_TET) else 1.0


# ----------------------------------------------------------------------------
# 1D
# ----------------------------------------------------------------------------

def gll_nodes(N: int) -> np.ndarray:
    """N+1 Gauss-Legendre-Lobatto points: -1, roots of P_N', +1."""
    interior = np.sort(npleg.Legendre.basis(N).deriv().roots().real)
    return np.concatenate([[-1.0], interior, [1.0]])


def gauss(q: int):
    return npleg.leggauss(q)


def lagrange_eval(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L[p, j] = ell_j(x_p) for the Lagrange basis on `nodes` (product form)."""
    x = np.atleast_1d(x)
    n = len(nodes)
    L = np.ones((x.size, n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_deriv(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dL[p, j] = ell_j'(x_p) by the product rule."""
    x = np.atleast_1d(x)
    n = len(nodes)
    D = np.zeros((x.size, n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            term = np.full(x.size, 1.0 / (nodes[j] - nodes[k]))
            for m in range(n):
                if m != j and m != k:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            D[:, j] += term
    return D


class Line:
    """1D reference element on GLL nodes."""

    def __init__(self, N: int):
        self.N = N
        self.x = gll_nodes(N)
        xq, wq = gauss(N + 3)
        Lq = lagrange_eval(self.x, xq)
        # M[i, j] = int ell_i ell_j
        self.M = Lq.T @ (wq[:, None] * Lq)
        # D[i, j] = ell_j'(x_i)
        self.D = lagrange_deriv(self.x, self.x)
        # GLL quadrature weights = integrals of the Lagrange basis
        self.w = Lq.T @ wq
        Minv = np.linalg.inv(self.M)
        self.ell0 = Minv[:, 0].copy()      # (M^1D)^{-1} e_0   (t = -1 face)
        self.ellN = Minv[:, N].copy()      # (M^1D)^{-1} e_N   (t = +1 face)
        # barycentric-weighted edge masses: int ell_i ell_j (1-x)/2, (1+x)/2
        self.Ma = Lq.T @ ((wq * (1 - xq) / 2)[:, None] * Lq)
        self.Mb = Lq.T @ ((wq * (1 + xq) / 2)[:, None] * Lq)


# ----------------------------------------------------------------------------
# warp & blend
# ----------------------------------------------------------------------------

def _warp(N: int, x: np.ndarray) -> np.ndarray:
    """Interpolant (on N+1 equispaced points) of the displacement that maps
    equispaced points to GLL points, divided by 1 - x^2 (zero at +-1)."""
    req = np.linspace(-1.0, 1.0, N + 1)
    disp = gll_nodes(N) - req
    w = lagrange_eval(req, x) @ disp
    out = np.zeros_like(w)
    inside = np.abs(x) < 1.0 - 1e-10
    out[inside] = w[inside] / (1.0 - x[inside] ** 2)
    return out


def _face_shift(N: int, alpha: float, L: np.ndarray, verts):
    """Barycentric displacement produced by the 2D warp of a triangle with
    vertices `verts` (indices into the columns of L).  Each edge (a, b) with
    opposite vertex c moves a point toward b by
        w = 4 L_a L_b warp(L_b - L_a) (1 + (alpha L_c)^2)
    measured in units where the edge has length 2, i.e. dL_b = w/2, dL_a = -w/2."""
    d = np.zeros_like(L)
    a0, a1, a2 = verts
    for (a, b, c) in ((a0, a1, a2), (a1, a2, a0), (a2, a0, a1)):
        w = 4.0 * L[:, a] * L[:, b] * _warp(N, L[:, b] - L[:, a]) * (1.0 + (alpha * L[:, c]) ** 2)
        d[:, b] += 0.5 * w
        d[:, a] -= 0.5 * w
    return d


@lru_cache(maxsize=None)
def tri_lattice(N: int):
    ab = [(a, b) for b in range(N + 1) for a in range(N + 1 - b)]
    return np.asarray(ab, dtype=np.int64)


@lru_cache(maxsize=None)
def tet_lattice(N: int):
    abc = [(a, b, c) for c in range(N + 1) for b in range(N + 1 - c) for a in range(N + 1 - b - c)]
    return np.asarray(abc, dtype=np.int64)


def tri_nodes(N: int) -> np.ndarray:
    """Triangle nodes (Nt, 2): 2D warp & blend with the tet blend parameter."""
    ab = tri_lattice(N)
    L = np.stack([(N - ab[:, 0] - ab[:, 1]) / N, ab[:, 0] / N, ab[:, 1] / N], axis=1)
    L = L + _face_shift(N, alpha_tet(N), L, (0, 1, 2))
    V = np.array([[-1.0, -1.0], [1.0, -1.0], [-1.0, 1.0]])
    return L @ V


def tet_nodes(N: int) -> np.ndarray:
    """Tetrahedron Warp & Blend nodes (Np, 3)."""
    abc = tet_lattice(N)
    lat = np.stack([N - abc.sum(axis=1), abc[:, 0], abc[:, 1], abc[:, 2]], axis=1)
    L = lat / N
    alpha = alpha_tet(N)
    shift = np.zeros_like(L)
    faces = ((3, (0, 1, 2)), (2, (0, 1, 3)), (0, (1, 2, 3)), (1, (0, 2, 3)))
    for (opp, fv) in faces:
        d = _face_shift(N, alpha, L, fv)
        La = L[:, opp]
        blend = L[:, fv[0]] * L[:, fv[1]] * L[:, fv[2]]
        denom = (L[:, fv[0]] + 0.5 * La) * (L[:, fv[1]] + 0.5 * La) * (L[:, fv[2]] + 0.5 * La)
        ok = denom > 1e-10
        blend[ok] = (1.0 + (alpha * La[ok]) ** 2) * blend[ok] / denom[ok]
        shift += blend[:, None] * d
    # points on tet edges take the pure 1D edge warp (the face blend above
    # degenerates there): reapply the warp of one face containing the edge
    nzero = (lat == 0).sum(axis=1)
    on_edge = nzero >= 2
    for (opp, fv) in faces:
        sel = on_edge & (lat[:, opp] == 0)
        if np.any(sel):
            shift[sel] = _face_shift(N, alpha, L[sel], fv)
    L = L + shift
    V = np.array([[-1.0, -1.0, -1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
    return L @ V


# ----------------------------------------------------------------------------
# quadrature on simplices (collapsed coordinates)
# ----------------------------------------------------------------------------

def tri_quadrature(q: int):
    """Duffy-collapsed Gauss rule on the bi-unit triangle, q x q points,
    exact for total degree <= 2q - 2."""
    x, w = gauss(q)
    A, B = np.meshgrid(x, x, indexing="ij")
    WA, WB = np.meshgrid(w, w, indexing="ij")
    r = (1 + A) * (1 - B) / 2 - 1
    s = B
    wt = WA * WB * (1 - B) / 2
    return np.stack([r.ravel(), s.ravel()], axis=1), wt.ravel()


def tet_quadrature(q: int):
    """Collapsed Gauss rule on the bi-unit tetrahedron, q^3 points,
    exact for total degree <= 2q - 3."""
    x, w = gauss(q)
    A, B, C = np.meshgrid(x, x, x, indexing="ij")
    WA, WB, WC = np.meshgrid(w, w, w, indexing="ij")
    r = (1 + A) * (1 - B) * (1 - C) / 4 - 1
    s = (1 + B) * (1 - C) / 2 - 1
    t = C
    wt = WA * WB * WC * (1 - B) * (1 - C) ** 2 / 8
    return np.stack([r.ravel(), s.ravel(), t.ravel()], axis=1), wt.ravel()


# ----------------------------------------------------------------------------
# Lagrange bases on simplices via a Legendre-product modal basis
# ----------------------------------------------------------------------------

def _legendre_all(N: int, x: np.ndarray):
    """P[k](x) and P'[k](x) for k = 0..N (standard Legendre)."""
    P = np.zeros((N + 1, x.size))
    dP = np.zeros((N + 1, x.size))
    for k in range(N + 1):
        c = np.zeros(k + 1)
        c[k] = 1.0
        P[k] = npleg.legval(x, c)
        dP[k] = npleg.legval(x, npleg.legder(c))
    return P, dP


def _modal2d(N: int, X: np.ndarray):
    """Values and r/s derivatives of P_a(r) P_b(s), a + b <= N."""
    r, s = X[:, 0], X[:, 1]
    Pr, dPr = _legendre_all(N, r)
    Ps, dPs = _legendre_all(N, s)
    idx = [(a, b) for a in range(N + 1) for b in range(N + 1 - a)]
    V = np.stack([Pr[a] * Ps[b] for a, b in idx], axis=1)
    Vr = np.stack([dPr[a] * Ps[b] for a, b in idx], axis=1)
    Vs = np.stack([Pr[a] * dPs[b] for a, b in idx], axis=1)
    return V, Vr, Vs


def _modal3d(N: int, X: np.ndarray):
    r, s, t = X[:, 0], X[:, 1], X[:, 2]
    Pr, dPr = _legendre_all(N, r)
    Ps, dPs = _legendre_all(N, s)
    Pt, dPt = _legendre_all(N, t)
    idx = [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a) for c in range(N + 1 - a - b)]
    V = np.stack([Pr[a] * Ps[b] * Pt[c] for a, b, c in idx], axis=1)
    Vr = np.stack([dPr[a] * Ps[b] * Pt[c] for a, b, c in idx], axis=1)
    Vs = np.stack([Pr[a] * dPs[b] * Pt[c] for a, b, c in idx], axis=1)
    Vt = np.stack([Pr[a] * Ps[b] * dPt[c] for a, b, c in idx], axis=1)
    return V, Vr, Vs, Vt


class Triangle:
    """Nodal triangle of degree N."""

    def __init__(self, N: int):
        self.N = N
        self.Nt = (N + 1) * (N + 2) // 2
        self.x = tri_nodes(N)                          # (Nt, 2)
        V, _, _ = _modal2d(N, self.x)
        self._Vinv = np.linalg.inv(V)
        # derivative matrices D[i, j] = d ell_j / dr (x_i)
        _, Vr, Vs = _modal2d(N, self.x)
        self.Dr = Vr @ self._Vinv
        self.Ds = Vs @ self._Vinv
        Xq, wq = tri_quadrature(N + 3)
        Lq = self.eval(Xq)
        self.M = Lq.T @ (wq[:, None] * Lq)
        lam = np.stack([-(Xq[:, 0] + Xq[:, 1]) / 2, (1 + Xq[:, 0]) / 2, (1 + Xq[:, 1]) / 2], axis=1)
        # barycentric-weighted masses  int ell_i ell_j lambda_a
        self.Ma = [Lq.T @ ((wq * lam[:, a])[:, None] * Lq) for a in range(3)]
        ab = tri_lattice(N)
        # edge node lists, ordered from the edge's first to its second vertex
        e0 = [i for i in range(self.Nt) if ab[i, 1] == 0]
        e0.sort(key=lambda i: ab[i, 0])
        e1 = [i for i in range(self.Nt) if ab[i, 0] + ab[i, 1] == N]
        e1.sort(key=lambda i: ab[i, 1])
        e2 = [i for i in range(self.Nt) if ab[i, 0] == 0]
        e2.sort(key=lambda i: -ab[i, 1])
        self.edges = [np.asarray(e) for e in (e0, e1, e2)]
        self.edge_vertices = ((0, 1), (1, 2), (2, 0))

    def eval(self, X: np.ndarray) -> np.ndarray:
        V, _, _ = _modal2d(self.N, X)
        return V @ self._Vinv

    def grad(self, X: np.ndarray):
        _, Vr, Vs = _modal2d(self.N, X)
        return Vr @ self._Vinv, Vs @ self._Vinv


class Tet:
    """Nodal tetrahedron of degree N."""

    # faces: (vertex triple, name); outward faces of the reference tet
    FACE_VERTS = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))

    def __init__(self, N: int):
        self.N = N
        self.Np = (N + 1) * (N + 2) * (N + 3) // 6
        self.x = tet_nodes(N)
        V, Vr, Vs, Vt = _modal3d(N, self.x)
        self._Vinv = np.linalg.inv(V)
        self.Dr = Vr @ self._Vinv
        self.Ds = Vs @ self._Vinv
        self.Dt = Vt @ self._Vinv
        Xq, wq = tet_quadrature(N + 3)
        Lq = self.eval(Xq)
        self.M = Lq.T @ (wq[:, None] * Lq)
        abc = tet_lattice(N)
        a, b, c = abc[:, 0], abc[:, 1], abc[:, 2]
        conds = (c == 0, b == 0, a + b + c == N, a == 0)
        self.faces = [np.nonzero(cnd)[0] for cnd in conds]

    def eval(self, X: np.ndarray) -> np.ndarray:
        V, _, _, _ = _modal3d(self.N, X)
        return V @ self._Vinv

    def grad(self, X: np.ndarray):
        _, Vr, Vs, Vt = _modal3d(self.N, X)
        return Vr @ self._Vinv, Vs @ self._Vinv, Vt @ self._Vinv


class Wedge:
    """Nodal wedge = triangle x GLL line; node n = j * Nt + i."""

    def __init__(self, N: int):
        self.N = N
        self.tri = Triangle(N)
        self.line = Line(N)
        self.Nt = self.tri.Nt
        self.Nq = N + 1
        self.Np = self.Nt * self.Nq
        I = np.repeat(np.arange(self.Nq), self.Nt)          # slice index j of node n
        Iv = np.tile(np.arange(self.Nt), self.Nq)            # triangle index i of node n
        self.node_j = I
        self.node_i = Iv
        self.x = np.stack([self.tri.x[Iv, 0], self.tri.x[Iv, 1], self.line.x[I]], axis=1)
        # faces: 0 bottom (t=-1), 1 top (t=+1), 2..4 quads over triangle edges 0..2
        self.faces = [np.arange(self.Nt), (self.Nq - 1) * self.Nt + np.arange(self.Nt)]
        for e in range(3):
            en = self.tri.edges[e]
            self.faces.append(np.asarray([j * self.Nt + en[m] for j in range(self.Nq) for m in range(self.Nq)]))

    def eval(self, X: np.ndarray) -> np.ndarray:
        Lt = self.tri.eval(X[:, :2])
        L1 = lagrange_eval(self.line.x, X[:, 2])
        return (L1[:, self.node_j] * Lt[:, self.node_i])

    def grad(self, X: np.ndarray):
        Ltr, Lts = self.tri.grad(X[:, :2])
        Lt = self.tri.eval(X[:, :2])
        L1 = lagrange_eval(self.line.x, X[:, 2])
        dL1 = lagrange_deriv(self.line.x, X[:, 2])
        j, i = self.node_j, self.node_i
        return (L1[:, j] * Ltr[:, i], L1[:, j] * Lts[:, i], dL1[:, j] * Lt[:, i])


def wedge_quadrature(q: int):
    Xt, wt = tri_quadrature(q)
    x1, w1 = gauss(q)
    X = np.array([[p[0], p[1], z] for z in x1 for p in Xt])
    W = np.array([wz * w for wz in w1 for w in wt])
    return X, W


@lru_cache(maxsize=None)
def wedge(N: int) -> Wedge:
    return Wedge(N)


@lru_cache(maxsize=None)
def tet(N: int) -> Tet:
    return Tet(N)


def wedge_vertex_functions(X: np.ndarray):
    """Bi-unit wedge vertex functions v_1..v_6 (Section 3.2 with the reference
    coordinates mapped from [0,1] to [-1,1]) and their gradients."""
    r, s, t = X[:, 0], X[:, 1], X[:, 2]
    lam = [-(r + s) / 2, (1 + r) / 2, (1 + s) / 2]
    dlam = [(-0.5, -0.5), (0.5, 0.0), (0.0, 0.5)]
    lo, hi = (1 - t) / 2, (1 + t) / 2
    v = np.stack([lam[0] * lo, lam[1] * lo, lam[2] * lo, lam[0] * hi, lam[1] * hi, lam[2] * hi], axis=1)
    g = np.zeros((X.shape[0], 6, 3))
    for a in range(3):
        for (col, tf, dtf) in ((a, lo, -0.5), (a + 3, hi, 0.5)):
            g[:, col, 0] = dlam[a][0] * tf
            g[:, col, 1] = dlam[a][1] * tf
            g[:, col, 2] = lam[a] * dtf
    return v, g


def tet_vertex_functions(X: np.ndarray):
    r, s, t = X[:, 0], X[:, 1], X[:, 2]
    v = np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2], axis=1)
    g = np.zeros((X.shape[0], 4, 3))
    g[:, 0, :] = -0.5
    g[:, 1, 0] = 0.5
    g[:, 2, 1] = 0.5
    g[:, 3, 2] = 0.5
    return v, g


LSRK45_A = (0.0,
            -567301805773.0 / 1357537059087.0,
            -2404267990393.0 / 2016746695238.0,
            -3550918686646.0 / 2091501179385.0,
            -1275806237668.0 / 842570457699.0)
LSRK45_B = (1432997174477.0 / 9575080441755.0,
            5161836677717.0 / 13612068292357.0,
            1720146321549.0 / 2090206949498.0,
            3134564353537.0 / 4481467310338.0,
            2277821191437.0 / 14882151754819.0)
LSRK45_C = (0.0,
            1432997174477.0 / 9575080441755.0,
            2526269341429.0 / 6820363962896.0,
            2006345519317.0 / 3224310063776.0,
            2802321613138.0 / 2924317926251.0)
"""Carpenter & Kennedy (1994) five-stage fourth-order 2N-storage Runge-Kutta
coefficients (their solution 3): res <- a_s res + dt f(t + c_s dt, q);
q <- q + b_s res."""


def nfaces(etype: int) -> int:
    return 5 if etype == 6 else 4

