"""Pins for the oracle's geometry (Lemma 3.1) and discrete operators
(Sections 2.1 and 4.2) against mathematics the paper fixes: the generic
vertex map, polynomial reproduction, discrete integration by parts,
Kronecker mass == brute-force mass, constant states and conservation."""
import numpy as np
import pytest

from oracle import reference as R
from oracle.dg import Solver
from paper_1607_03399_gb300 import inputs as I


def _random_vertical_wedge(rng):
    """A vertically mapped wedge with a skewed footprint and tilted, non-parallel
    top and bottom faces."""
    xy = np.array([[0.0, 0.0], [1.0, 0.2], [0.3, 0.9]]) + rng.uniform(-0.1, 0.1, (3, 2))
    zb = rng.uniform(-0.2, 0.2, 3)
    zt = 1.0 + rng.uniform(-0.3, 0.3, 3)
    V = np.zeros((6, 3))
    V[:3, :2] = xy
    V[3:, :2] = xy
    V[:3, 2] = zb
    V[3:, 2] = zt
    return V


def test_lemma_3_1_against_generic_jacobian():
    """J constant in t, r_z = s_z = 0, r_x..s_y and t_z J constant, t_x J and
    t_y J linear in t: checked against the generic vertex-map Jacobian."""
    rng = np.random.default_rng(7)
    N = 3
    for _ in range(5):
        V = _random_vertical_wedge(rng)
        S = Solver(V, np.arange(6)[None, :], np.array([6], dtype=np.uint8), N)
        g = S.wg
        X = np.column_stack([rng.uniform(-1, 0, 20), rng.uniform(-1, 0, 20), rng.uniform(-1, 1, 20)])
        X[:, 1] = np.minimum(X[:, 1], -X[:, 0])      # inside the triangle
        _, gv = R.wedge_vertex_functions(X)
        G = np.einsum("qvm,vd->qdm", gv, V)           # dx_d / dr_m
        J = np.linalg.det(G)
        Gi = np.linalg.inv(G)                         # dr_m / dx_d
        lam = np.stack([-(X[:, 0] + X[:, 1]) / 2, (1 + X[:, 0]) / 2, (1 + X[:, 1]) / 2], axis=1)
        assert np.allclose(J, lam @ g["Ja"][0], rtol=1e-13)       # J linear in r,s, no t
        assert np.allclose(Gi[:, 0, 2], 0, atol=1e-13)              # r_z
        assert np.allclose(Gi[:, 1, 2], 0, atol=1e-13)              # s_z
        assert np.allclose(Gi[:, 0, 0], g["rx"][0]) and np.allclose(Gi[:, 0, 1], g["ry"][0])
        assert np.allclose(Gi[:, 1, 0], g["sx"][0]) and np.allclose(Gi[:, 1, 1], g["sy"][0])
        assert np.allclose(Gi[:, 2, 2] * J, g["A"][0])              # t_z J = A
        # t_x J, t_y J: linear in t, equal to the closed form at the GLL points
        t = S.W.line.x
        for comp, key in ((0, "txJ"), (1, "tyJ")):
            vals = Gi[:, 2, comp] * J
            coef = np.polyfit(t, g[key][0], 1)
            assert np.allclose(np.polyval(coef, X[:, 2]), vals, atol=1e-12)
        # volume and face areas by the generic map
        Xq, wq = R.wedge_quadrature(4)
        _, gq = R.wedge_vertex_functions(Xq)
        vol = wq @ np.linalg.det(np.einsum("qvm,vd->qdm", gq, V))
        assert abs(vol - g["vol"][0]) < 1e-13


def test_mesh_volume_sums_to_domain():
    mesh = I.cube_wavy_mesh(4, 4, 0.03)
    S = Solver(mesh.VX, mesh.EToV, mesh.etype, 2)
    assert abs(S.wg["vol"].sum() - 1.0) < 1e-13
    hm = I.hybrid_mesh(3, 2, 2)
    S2 = Solver(hm.VX, hm.EToV, hm.etype, 1)
    assert abs(S2.wg["vol"].sum() + S2.tg["vol"].sum() - 1.0) < 1e-13


MESHES = {
    "wavy": lambda: I.cube_wavy_mesh(2, 2, 0.05),
    "perturbed": lambda: I.perturbed_layered_mesh(2, 2, 0.3, 1),
    "hybrid": lambda: I.hybrid_mesh(2, 1, 1),
    "tets": lambda: I.tet_box_mesh(1, 1),
}


@pytest.mark.parametrize("meshname", list(MESHES))
@pytest.mark.parametrize("N", [1, 2, 3])
@pytest.mark.parametrize("bc,flux", [("rigid", "upwind"), ("dirichlet", "central")])
def test_method_form_equals_brute_force(meshname, N, bc, flux):
    """Section 4.2's Kronecker/Lemma 3.1 form reproduces the plain
    exact-quadrature definition of Section 2.1 (random state, random
    piecewise-constant rho and c)."""
    mesh = MESHES[meshname]()
    c2, rho = I.random_material(mesh.K, 11, 1.0, 3.0, 0.5, 2.0)
    S = Solver(mesh.VX, mesh.EToV, mesh.etype, N, c2, rho, bc=bc, flux=flux)
    q = I.random_fields(S.conn.total_nodes, 5)
    a, b = S.rhs(q), S.rhs_brute(q)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)


@pytest.mark.parametrize("meshname", ["wavy", "perturbed", "hybrid", "tets"])
@pytest.mark.parametrize("N", [1, 2, 3])
def test_polynomial_exactness_gradient_divergence(meshname, N):
    """Vertex-mapped elements reproduce total-degree-N polynomials (Section 3),
    so for a global polynomial the interior jumps vanish and the RHS is the
    exact derivative: rigid walls, u=0  -> rhs_u = -grad p / rho;
    Dirichlet, p=0 -> rhs_p = -kappa div u."""
    mesh = MESHES[meshname]()
    rng = np.random.default_rng(N)
    K = mesh.K
    c2, rho = np.full(K, 2.0), np.full(K, 0.5)
    S = Solver(mesh.VX, mesh.EToV, mesh.etype, N, c2, rho, bc="rigid")
    x, y, z = S.conn.xyz
    mons = [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a) for c in range(N + 1 - a - b)]
    coef = rng.normal(size=len(mons))
    f = sum(cf * x ** a * y ** b * z ** c for cf, (a, b, c) in zip(coef, mons))
    df = [sum(cf * a * x ** max(a - 1, 0) * y ** b * z ** c for cf, (a, b, c) in zip(coef, mons)),
          sum(cf * b * x ** a * y ** max(b - 1, 0) * z ** c for cf, (a, b, c) in zip(coef, mons)),
          sum(cf * c * x ** a * y ** b * z ** max(c - 1, 0) for cf, (a, b, c) in zip(coef, mons))]
    q = np.zeros((4, S.conn.total_nodes))
    q[0] = f
    r = S.rhs(q)
    scale = max(1.0, np.abs(df).max())
    for c in range(3):
        assert np.allclose(r[1 + c], -df[c] / 0.5, atol=1e-10 * scale)
    assert np.allclose(r[0], 0, atol=1e-10 * scale)
    S2 = Solver(mesh.VX, mesh.EToV, mesh.etype, N, c2, rho, bc="dirichlet")
    q = np.zeros((4, S.conn.total_nodes))
    q[1], q[2], q[3] = f, 2 * f, -f
    r = S2.rhs(q)
    div = df[0] + 2 * df[1] - df[2]
    assert np.allclose(r[0], -1.0 * div, atol=1e-10 * scale)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_discrete_integration_by_parts(N):
    """S_x + S_x^T = sum_f n_x M_f on every element (exact quadrature);
    Kronecker mass M^tri (x) M^1D equals the brute-force mass."""
    mesh = I.perturbed_layered_mesh(2, 1, 0.3, 2)
    hm = I.hybrid_mesh(1, 1, 1)
    for m in (mesh, hm):
        S = Solver(m.VX, m.EToV, m.etype, N)
        Ms = S.element_mass_method()
        for k in range(S.K):
            M, Sd, faces = S.element_matrices(k)
            Np = M.shape[0]
            assert np.allclose(Ms[k], M, atol=1e-13 * np.abs(M).max())
            for d in range(3):
                B = np.zeros((Np, Np))
                for (fn, Mf, nrm) in faces:
                    B[:, fn] += nrm[d] * Mf
                assert np.allclose(Sd[d] + Sd[d].T, B, atol=1e-12)


def test_affine_wedge_triangular_lift_is_scaled_identity():
    """If the wedge is affine (equal column heights), L^tri = (M^tri)^{-1}
    M^tri_hat reduces to I / J (Section 4.2)."""
    V = _random_vertical_wedge(np.random.default_rng(3))
    V[3:, 2] = V[:3, 2] + 0.7
    S = Solver(V, np.arange(6)[None, :], np.array([6], dtype=np.uint8), 3)
    Lt = np.linalg.solve(S.wedge_tri_mass()[0], S.W.tri.M)
    J = S.wg["Ja"][0, 0]
    assert np.allclose(Lt, np.eye(S.W.Nt) / J, atol=1e-12)


@pytest.mark.parametrize("meshname", ["wavy", "hybrid"])
def test_constant_state_and_conservation(meshname):
    mesh = MESHES[meshname]()
    c2, rho = I.random_material(mesh.K, 4, 1.0, 2.0, 1.0, 3.0)
    S = Solver(mesh.VX, mesh.EToV, mesh.etype, 3, c2, rho, bc="rigid")
    q = np.zeros((4, S.conn.total_nodes))
    q[0] = 2.5
    assert np.abs(S.rhs(q)).max() < 1e-11
    # int p / kappa is conserved under rigid walls for any state
    q = I.random_fields(S.conn.total_nodes, 9)
    r = S.rhs(q)
    Ms = S.element_mass_method()
    C = S.conn
    tot = sum(np.ones(C.offset[k + 1] - C.offset[k]) @ Ms[k] @ r[0, C.offset[k]:C.offset[k + 1]] / S.kappa[k]
              for k in range(S.K))
    assert abs(tot) < 1e-11 * np.abs(r).max()


def test_stable_dt_formula():
    mesh = I.cube_wavy_mesh(4, 4, 0.0)
    S = Solver(mesh.VX, mesh.EToV, mesh.etype, 3)
    # flat layers: largest face/volume ratio is the quad face of the right
    # triangle with legs 1/4: area (sqrt2/4)(1/4), volume (1/32)(1/4)
    ratio = (np.sqrt(2) / 16) / (1 / 128)
    assert abs(S.stable_dt(0.5) - 0.5 / (16 * ratio)) < 1e-14


def test_point_source_is_the_weak_delta():
    """The source vector g = kappa M^{-1} l(x_s) satisfies v^T M g / kappa = v(x_s)
    for every v in the element space (the weak form of a point load), and the
    Ricker wavelet has its closed-form peak and zeros."""
    m = I.cube_wavy_mesh(2, 2, 0.05)
    S = Solver(m.VX, m.EToV, m.etype, 3, np.full(m.K, 2.0), np.full(m.K, 0.5))
    k = S.add_source(0.3, 0.6, 0.45, 10.0, 0.1, 1.0)
    _, g, _, _, _ = S.sources[0]
    M, _, _ = S.element_matrices(k)
    X = S.reference_coords(k, (0.3, 0.6, 0.45))
    xyz = S.conn.xyz[:, S.conn.offset[k]:S.conn.offset[k + 1]]
    for v in (np.ones(xyz.shape[1]), xyz[0] ** 2 - xyz[2], xyz[1] * xyz[2] ** 3):
        val = S.W.eval(X[None, :])[0] @ v
        assert abs(v @ M @ g / S.kappa[k] - val) < 1e-12
    assert abs(S.ricker(10.0, 0.0) - 1.0) < 1e-15
    tz = 1.0 / (np.sqrt(2.0) * np.pi * 10.0)
    assert abs(S.ricker(10.0, tz)) < 1e-15
    # the source enters only the pressure rows of its element
    q = np.zeros((4, S.conn.total_nodes))
    r = S.rhs(q, t=0.1)
    assert np.count_nonzero(r[1:]) == 0
    assert np.allclose(r[0, S.conn.offset[k]:S.conn.offset[k + 1]], g)
