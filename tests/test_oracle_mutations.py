"""The oracle's pins are sensitive: each plausible mistake planted here (in a
private copy of the oracle's data, on the CPU) is caught by the pin that
guards it."""
import copy

import numpy as np

from oracle.dg import Solver
from paper_1607_03399_gb300 import inputs as I


def _setup(N=2, bc="rigid", flux="upwind"):
    m = I.perturbed_layered_mesh(2, 2, 0.3, 1)
    c2, rho = I.random_material(m.K, 2, 1.0, 3.0, 0.5, 2.0)
    S = Solver(m.VX, m.EToV, m.etype, N, c2, rho, bc=bc, flux=flux)
    S.W = copy.deepcopy(S.W)
    return S


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_dropped_t_derivative_term_is_caught():
    S = _setup()
    q = I.random_fields(S.conn.total_nodes, 1)
    ref = S.rhs_brute(q)
    assert _rel(S.rhs(q), ref) < 1e-13
    S.wg["txJ"] = np.zeros_like(S.wg["txJ"])
    assert _rel(S.rhs(q), ref) > 1e-3


def test_lumped_jacobian_weight_is_caught():
    """Replacing M^{tri,k} = sum_a J_a M_a by (mean J) M_hat (a plausible
    simplification) breaks agreement with the exact-quadrature definition."""
    S = _setup()
    q = I.random_fields(S.conn.total_nodes, 2)
    ref = S.rhs_brute(q)
    Ja = S.wg["Ja"].mean(axis=1, keepdims=True)
    S.wg["Ja"] = np.repeat(Ja, 3, axis=1)
    assert _rel(S.rhs(q), ref) > 1e-3


def test_swapped_tri_face_lift_is_caught():
    S = _setup()
    q = I.random_fields(S.conn.total_nodes, 3)
    ref = S.rhs_brute(q)
    S.W.line.ell0, S.W.line.ellN = S.W.line.ellN.copy(), S.W.line.ell0.copy()
    assert _rel(S.rhs(q), ref) > 1e-3


def test_flipped_quad_normal_breaks_energy_identity():
    S = _setup(flux="central")
    q = I.random_fields(S.conn.total_nodes, 4)
    Wm = S.energy_weights()
    E = 0.5 * q.ravel() @ Wm @ q.ravel()
    assert abs(q.ravel() @ Wm @ S.rhs(q).ravel()) < 1e-12 * E
    S.wg["n_quad"] = -S.wg["n_quad"]
    assert abs(q.ravel() @ Wm @ S.rhs(q).ravel()) > 1e-6 * E


def test_wrong_penalty_average_is_caught():
    """tau from the interior side only instead of {rho c}: the energy identity
    with the averaged penalty no longer holds on a mesh with jumps in rho c."""
    S = _setup(flux="upwind")
    q = I.random_fields(S.conn.total_nodes, 5)
    Wm = S.energy_weights()
    diss = S.face_dissipation(q)
    assert abs(q.ravel() @ Wm @ S.rhs(q).ravel() - diss) < 1e-12 * abs(diss)
    orig = S.face_flux

    def one_sided(q_, typ, f, normal):
        saved = S.rhoc.copy()
        gM, gP, nbr = S.ftab[(typ, f)]
        elems = S.conn.wedges if typ == 6 else S.conn.tets
        S.rhoc = saved.copy()
        S.rhoc[nbr[nbr >= 0]] = saved[elems[nbr >= 0]]
        try:
            return orig(q_, typ, f, normal)
        finally:
            S.rhoc = saved
    S.face_flux = one_sided
    assert abs(q.ravel() @ Wm @ S.rhs(q).ravel() - diss) > 1e-6 * abs(diss)
