"""Oracle pins for the adjoint (CPU).

* The method's operator is skew-adjoint in the energy inner product apart from
  the symmetric upwind penalty (Section 4.1: the central flux conserves the
  discrete energy, the penalty only dissipates), so A^T = W P A P W^{-1} with W
  the energy mass and P = diag(1, -I) flipping the velocity.  Checked on dense
  matrices for both fluxes and both walls, wedge and hybrid meshes.
* The oracle's reverse-mode gradient of the receiver misfit equals central
  differences of the misfit."""
import numpy as np
import pytest

from oracle import adjoint as OA
from oracle.dg import Solver as Oracle
from paper_1607_03399_gb300 import inputs as I


@pytest.mark.parametrize("meshname", ["wedges", "hybrid"])
@pytest.mark.parametrize("bc,flux", [("rigid", "upwind"), ("dirichlet", "upwind"), ("rigid", "central"),
                                     ("dirichlet", "central")])
def test_transpose_is_energy_weighted_velocity_flip(meshname, bc, flux):
    m = I.perturbed_layered_mesh(2, 2, 0.2, 0) if meshname == "wedges" else I.hybrid_mesh(2, 1, 1)
    c2, rho = I.random_material(m.K, 4, 1.0, 2.5, 0.6, 1.4)
    O = Oracle(m.VX, m.EToV, m.etype, 2, c2, rho, bc=bc, flux=flux)
    A = O.dense_A()
    W = O.energy_weights()
    n = O.conn.total_nodes
    P = np.ones(4 * n)
    P[n:] = -1.0
    rhs = W @ (P[:, None] * A * P[None, :]) @ np.linalg.inv(W)
    assert np.abs(A.T - rhs).max() <= 1e-11 * np.abs(A).max()
    # and the relation is not empty: A itself is far from its transpose
    assert np.abs(A.T - A).max() > 1e-2 * np.abs(A).max()


@pytest.mark.parametrize("meshname", ["wedges", "hybrid"])
def test_oracle_reverse_gradient_matches_finite_differences(meshname):
    m = I.cube_wavy_mesh(2, 1, 0.05) if meshname == "wedges" else I.hybrid_mesh(2, 1, 1)
    rng = np.random.default_rng(0)
    kap, rho = rng.uniform(1, 2, m.K), rng.uniform(0.8, 1.3, m.K)
    st = OA.Setup(m, 1, kap, rho, [(0.4, 0.6, 0.5, 3.0, 0.2, 1.0)], [(0.7, 0.3, 0.6), (0.2, 0.2, 0.3)], 0.02, 12)
    data = OA.traces(st) * 0.9 + 0.01
    gk, gr = OA.gradient_reverse(st, data)
    # wedges and, on the hybrid mesh, tets on both sides of the interface
    picks = (0, 3, 7) if meshname == "wedges" else (0, 7, 8, 20, m.K - 1)
    fk, fr = OA.gradient_fd(st, data, list(picks))
    for k in picks:
        assert abs(gk[k] - fk[k]) <= 1e-6 * abs(fk[k])
        assert abs(gr[k] - fr[k]) <= 1e-6 * abs(fr[k])
