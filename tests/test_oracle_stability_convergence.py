"""Pins for energy stability (Section 4.1, eq. (2), Figs 2-3) and accuracy
(Section 6.1, Table 1) of the oracle."""
import json
import os

import numpy as np
import pytest

from oracle.dg import Solver
from paper_1607_03399_gb300 import inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_rates.json")))


@pytest.mark.parametrize("bc", ["rigid", "dirichlet"])
@pytest.mark.parametrize("flux", ["upwind", "central"])
@pytest.mark.parametrize("N", [1, 2, 3])
def test_semidiscrete_energy_identity(bc, flux, N):
    """dE/dt = q^T W rhs(q) equals the face dissipation
    -1/2 sum_interior int (tau_p [p]^2 + tau_u [u_n]^2) - 1/4 sum_boundary (...)
    (zero for the central flux) -- the identity behind eq. (2)."""
    mesh = I.hybrid_mesh(2, 1, 1)
    c2, rho = I.random_material(mesh.K, 3, 1.0, 3.0, 0.5, 2.0)
    S = Solver(mesh.VX, mesh.EToV, mesh.etype, N, c2, rho, bc=bc, flux=flux)
    q = I.random_fields(S.conn.total_nodes, 21)
    Wm = S.energy_weights()
    dE = q.ravel() @ Wm @ S.rhs(q).ravel()
    diss = S.face_dissipation(q)
    E = 0.5 * q.ravel() @ Wm @ q.ravel()
    assert abs(E - S.energy(q)) < 1e-12 * E
    if flux == "central":
        assert diss == 0.0
        assert abs(dE) < 1e-12 * E
    else:
        assert diss < 0
        assert abs(dE - diss) < 1e-12 * abs(diss)


def _spectrum_mesh():
    # 2x2 squares -> 8 triangles, 2 layers = 16 wedges on the bi-unit cube;
    # interior interface moved vertically by U(-0.25, 0.25) layer heights
    return I.perturbed_layered_mesh(2, 2, 0.25, 0)


@pytest.mark.parametrize("flux", ["upwind", "central"])
def test_spectrum_exact_mass_is_stable(flux):
    """Fig. 3: with the exact (Jacobian-weighted) wedge mass every eigenvalue of
    the DG operator has non-positive real part up to machine precision."""
    m = _spectrum_mesh()
    S = Solver(m.VX, m.EToV, m.etype, 2, bc="dirichlet", flux=flux)
    lam = np.linalg.eigvals(S.dense_A())
    assert lam.real.max() <= 1e-10 * np.abs(lam).max()
    if flux == "upwind":
        assert lam.real.min() < -1.0          # genuinely dissipative


@pytest.mark.parametrize("flux", ["upwind", "central"])
def test_spectrum_mass_lumping_is_unstable(flux):
    """Fig. 2: GLL mass lumping in t (which changes only the triangle-face
    lift and the mass norm for vertically mapped wedges) yields eigenvalues
    with positive real part."""
    m = _spectrum_mesh()
    S = Solver(m.VX, m.EToV, m.etype, 2, bc="dirichlet", flux=flux, lumped=True)
    lam = np.linalg.eigvals(S.dense_A())
    assert lam.real.max() > 1e-3


def test_fully_discrete_energy_decay():
    """128-wedge wavy cube, N=3, upwind, rigid walls, LSRK45 at CFL 0.5: the
    discrete energy never increases over 200 steps."""
    m = I.cube_wavy_mesh(4, 4, 0.03)
    S = Solver(m.VX, m.EToV, m.etype, 3, bc="rigid", flux="upwind")
    q = I.standing_mode_unit_cube(S.conn.xyz, 0.0)
    dt = S.stable_dt(0.5)
    E = [S.energy(q)]
    for _ in range(20):
        q = S.step(q, dt, 10)
        E.append(S.energy(q))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-14 * E[0])
    assert E[-1] < E[0]


def _rate(N, ms, mesh_fn, exact, bc, T):
    errs = []
    for m in ms:
        mesh = mesh_fn(m)
        S = Solver(mesh.VX, mesh.EToV, mesh.etype, N, bc=bc, flux="upwind")
        q0 = exact(S.conn.xyz, 0.0)
        n = int(np.ceil(T / S.stable_dt(0.5)))
        q = S.step(q0, T / n, n)
        e = S.l2_error(q, exact, T)
        errs.append(np.sqrt((e ** 2).sum()))
    return np.log2(errs[0] / errs[1]), errs


@pytest.mark.parametrize("N,ms", [(1, (4, 8)), (2, (2, 4)), (3, (2, 4))])
def test_convergence_rigid_unit_cube(N, ms):
    """Rigid-wall standing mode on wavy layered meshes of the unit cube:
    observed rate ~ N+1, within 0.35 of the structured rates of Table 1."""
    rate, errs = _rate(N, ms, lambda m: I.cube_wavy_mesh(m, m, 0.03), I.standing_mode_unit_cube, "rigid", 0.3)
    assert abs(rate - GOLDEN["table1_rates"]["structured"][str(N)]) < 0.35, (rate, errs)


@pytest.mark.parametrize("N", [2, 3])
def test_convergence_dirichlet_perturbed_biunit_cube(N):
    """Homogeneous-Dirichlet mode of Section 6.1 on randomly perturbed
    (non-nested) vertically mapped meshes of the bi-unit cube: rate near N+1
    (Table 1, unstructured: 2.9 and 4.42)."""
    rate, errs = _rate(N, (2, 4), lambda m: I.perturbed_layered_mesh(m, m, 0.2, 100 + m),
                       I.standing_mode_biunit_cube, "dirichlet", 0.5)
    assert N + 0.5 < rate < N + 2.0, (rate, errs)
