"""Pins for the oracle's reference elements (Section 3.1 and 4.2 of the paper)
against closed forms: GLL points, exact integrals of barycentric monomials,
exact derivatives of polynomials, node-set symmetry and conformity."""
import itertools
import math

import numpy as np
import pytest

from oracle import reference as R


@pytest.mark.parametrize("N,expected", [
    (1, [-1.0, 1.0]),
    (2, [-1.0, 0.0, 1.0]),
    (3, [-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0]),
    (4, [-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0]),
])
def test_gll_closed_form(N, expected):
    assert np.allclose(R.gll_nodes(N), expected, atol=1e-14)


def _bary_tri(X):
    r, s = X[:, 0], X[:, 1]
    return np.stack([-(r + s) / 2, (1 + r) / 2, (1 + s) / 2], axis=1)


def _bary_tet(X):
    r, s, t = X[:, 0], X[:, 1], X[:, 2]
    return np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2], axis=1)


def _tri_int(powers):
    """int over the bi-unit triangle (area 2) of prod lambda_i^a_i."""
    a = list(powers)
    return 2 * 2 * math.prod(math.factorial(x) for x in a) / math.factorial(sum(a) + 2)


def _tet_int(powers):
    """int over the bi-unit tet (volume 4/3) of prod lambda_i^a_i."""
    a = list(powers)
    return 6 * (4 / 3) * math.prod(math.factorial(x) for x in a) / math.factorial(sum(a) + 3)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_line_mass_derivative_lift(N):
    L = R.Line(N)
    x = L.x
    for a in range(N + 1):
        for b in range(N + 1):
            exact = (1 - (-1) ** (a + b + 1)) / (a + b + 1)
            assert abs(x ** a @ L.M @ x ** b - exact) < 1e-13
            # (1-x)/2 weight: int x^(a+b) (1-x)/2
            ex_a = 0.5 * (exact - (1 - (-1) ** (a + b + 2)) / (a + b + 2))
            assert abs(x ** a @ L.Ma @ x ** b - ex_a) < 1e-13
        d = a * x ** (a - 1) if a > 0 else np.zeros_like(x)
        assert np.allclose(L.D @ x ** a, d, atol=1e-12)
        # lift vectors: f^T M ell0 = f(-1), f^T M ellN = f(1)
        assert abs(x ** a @ L.M @ L.ell0 - (-1.0) ** a) < 1e-12
        assert abs(x ** a @ L.M @ L.ellN - 1.0) < 1e-12
    assert abs(L.w.sum() - 2) < 1e-14


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_triangle_mass_and_weighted_masses(N):
    T = R.Triangle(N)
    lam = _bary_tri(T.x)
    assert abs(T.M.sum() - 2) < 1e-12
    assert np.all(np.linalg.eigvalsh(T.M) > 0)
    # f, g total degree <= N (barycentric monomials): f^T M g = int f g
    pw = [p for p in itertools.product(range(N + 1), repeat=2) if sum(p) <= N]
    for (a, b) in pw[:6]:
        for (c, d) in pw[-4:]:
            f = lam[:, 1] ** a * lam[:, 2] ** b
            g = lam[:, 0] ** c * lam[:, 1] ** d
            ex = _tri_int((c, a + d, b))
            assert abs(f @ T.M @ g - ex) < 1e-12
            for k in range(3):
                pk = [c, a + d, b]
                pk[k] += 1
                assert abs(f @ T.Ma[k] @ g - _tri_int(pk)) < 1e-12
    assert np.allclose(sum(T.Ma), T.M, atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_triangle_derivatives_exact(N):
    T = R.Triangle(N)
    r, s = T.x[:, 0], T.x[:, 1]
    for a in range(N + 1):
        for b in range(N + 1 - a):
            f = r ** a * s ** b
            fr = a * r ** max(a - 1, 0) * s ** b if a else np.zeros_like(r)
            fs = b * r ** a * s ** max(b - 1, 0) if b else np.zeros_like(r)
            assert np.allclose(T.Dr @ f, fr, atol=1e-11)
            assert np.allclose(T.Ds @ f, fs, atol=1e-11)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_tet_mass_and_derivatives(N):
    T = R.Tet(N)
    lam = _bary_tet(T.x)
    assert abs(T.M.sum() - 4 / 3) < 1e-12
    assert np.all(np.linalg.eigvalsh(T.M) > 0)
    for (a, b, c) in [(N, 0, 0), (0, N, 0), (1, 0, N - 1), (0, 0, 0)]:
        f = lam[:, 1] ** a * lam[:, 2] ** b * lam[:, 3] ** c
        g = lam[:, 0] ** N
        assert abs(f @ T.M @ g - _tet_int((N, a, b, c))) < 1e-12
    r, s, t = T.x.T
    for (a, b, c) in [(N, 0, 0), (0, N, 0), (0, 0, N), (N - 1, 1, 0), (0, N - 1, 1) if N > 1 else (0, 0, 1)]:
        f = r ** a * s ** b * t ** c
        fr = a * r ** max(a - 1, 0) * s ** b * t ** c
        fs = b * r ** a * s ** max(b - 1, 0) * t ** c
        ft = c * r ** a * s ** b * t ** max(c - 1, 0)
        assert np.allclose(T.Dr @ f, fr, atol=1e-11)
        assert np.allclose(T.Ds @ f, fs, atol=1e-11)
        assert np.allclose(T.Dt @ f, ft, atol=1e-11)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_triangle_nodes_structure(N):
    """Vertices present, edge nodes are the GLL points, and the node set is
    invariant under the six symmetries of the triangle (needed for face
    orientation matching)."""
    T = R.Triangle(N)
    gll = R.gll_nodes(N)
    lam = _bary_tri(T.x)
    for e, (a, b) in enumerate(T.edge_vertices):
        en = T.edges[e]
        # parameter along the edge from vertex a (-1) to vertex b (+1)
        sigma = lam[en, b] - lam[en, a]
        assert np.allclose(sigma, gll, atol=1e-13)
    for perm in itertools.permutations(range(3)):
        P = lam[:, list(perm)]
        d = np.linalg.norm(P[:, None, :] - lam[None, :, :], axis=2)
        assert np.all(d.min(axis=1) < 1e-13)
    if N == 3:
        interior = [i for i in range(T.Nt) if np.all(lam[i] > 1e-12)]
        assert len(interior) == 1 and np.allclose(lam[interior[0]], 1 / 3, atol=1e-14)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_tet_faces_are_triangle_nodes(N):
    """Tet face nodes equal the triangle nodes mapped by the face vertices
    (wedge/tet conformity, Section 3.1)."""
    T = R.Tet(N)
    tri = R.Triangle(N)
    lt = _bary_tri(tri.x)
    tv = np.array([[-1.0, -1, -1], [1.0, -1, -1], [-1.0, 1, -1], [-1.0, -1, 1]])
    for f, fv in enumerate(R.Tet.FACE_VERTS):
        X = lt @ tv[list(fv)]
        assert np.allclose(T.x[T.faces[f]], X, atol=1e-13)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_wedge_tensor_structure(N):
    W = R.Wedge(N)
    assert W.Np == (N + 1) ** 2 * (N + 2) // 2
    assert len(W.faces) == 5
    # node n = j*Nt + i
    assert np.allclose(W.x[:W.Nt, :2], W.tri.x)
    assert np.allclose(W.x[::W.Nt, 2], W.line.x)
    # face node sets lie on their faces
    assert np.allclose(W.x[W.faces[0], 2], -1)
    assert np.allclose(W.x[W.faces[1], 2], 1)
    assert np.allclose(W.x[W.faces[2], 1], -1)
    assert np.allclose(W.x[W.faces[3], 0] + W.x[W.faces[3], 1], 0, atol=1e-14)
    assert np.allclose(W.x[W.faces[4], 0], -1)


def test_lsrk45_coefficients_fourth_order():
    """Carpenter-Kennedy LSRK45 is fourth order: error ratio ~16 on halving dt
    for y' = lam y."""
    from oracle.dg import lsrk45
    lam = -0.5 + 3.0j
    errs = []
    for n in (20, 40, 80):
        y = lsrk45(lambda q: lam * q, np.array([1.0 + 0j]), 2.0 / n, n)
        errs.append(abs(y[0] - np.exp(2.0 * lam)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 4.0) < 0.15), rates
    # consistency conditions of the 2N-storage scheme
    c = R.LSRK45_C
    assert abs(c[1] - R.LSRK45_B[0]) < 1e-15
    assert R.LSRK45_A[0] == 0.0
