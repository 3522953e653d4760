"""The allocation-free energy entry point, dg_energy_static.

Some callers cannot allocate device memory at the moment they need a
diagnostic: a framework may forbid allocations while it holds its memory
pool, and host callbacks may not allocate at all.  dg_energy_static computes
the discrete energy of a caller-provided state with its scratch in a
fixed-size array that the library owns, so it allocates nothing.  This test
calls it through the C ABI and checks it against dg_energy (which uses
scratch inside the caller-allocated mesh blob) on two calls in a row, against
the oracle's energy, and with two shots in both shot orders (a
[shots][4][total_nodes] state, energy summed over the shots).

The file is named to be collected last, so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

from oracle.dg import Solver as Oracle
from paper_1607_03399_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_1607_03399_gb300 import dg  # noqa: E402
from paper_1607_03399_gb300.dg import Solver  # noqa: E402


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-6)])
@pytest.mark.parametrize("meshname,N", [("hybrid", 3), ("wavy", 2), ("wavy", 4)])
def test_energy_static_matches_energy(precision, tol, meshname, N):
    m = I.hybrid_mesh(3, 2, 1) if meshname == "hybrid" else I.cube_wavy_mesh(4, 4, 0.03)
    c2, rho = I.random_material(m.K, 7, 1.0, 3.0, 0.5, 2.0)
    S = Solver(m.VX, m.EToV, m.etype, N, c2, rho, precision=precision)
    try:
        for seed in (1, 2):
            q = I.random_fields(S.total_nodes, seed).astype(S.np_dtype)
            S.set_fields(q)
            E_ref = dg.dg_energy(S.ctx)
            dq = torch.from_numpy(q).to(S.device)
            torch.cuda.synchronize(S.device)
            E1 = dg.dg_energy_static(S.ctx, dq.data_ptr())
            E2 = dg.dg_energy_static(S.ctx, dq.data_ptr())
            assert abs(E1 - E_ref) <= tol * E_ref, (E1, E_ref)
            assert abs(E2 - E_ref) <= tol * E_ref, (E2, E_ref)
            # the oracle's energy of the same (rounded) state
            E_or = Oracle(m.VX, m.EToV, m.etype, N, c2, rho).energy(q.astype(np.float64))
            assert abs(E1 - E_or) <= tol * E_or, (E1, E_or)
    finally:
        S.close()


@pytest.mark.parametrize("order", ["outer", "inner"])
@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_energy_static_sums_shots(order, precision, tol):
    """Two shots: the [shots][4][total_nodes] state's energy is the sum of the
    shots' energies (each from the oracle), on two calls in a row, and equals
    dg_energy of the bound two-shot state."""
    m = I.hybrid_mesh(3, 2, 1)
    c2, rho = I.random_material(m.K, 5, 1.0, 3.0, 0.5, 2.0)
    S = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision=precision, shots=2, shot_order=order)
    O = Oracle(m.VX, m.EToV, m.etype, 3, c2, rho)
    try:
        rng = np.random.default_rng(11)
        q = rng.uniform(-1, 1, size=(2, 4, S.total_nodes)).astype(S.np_dtype)
        q[1] *= 0.5  # shots of different size
        E_or = sum(O.energy(q[s].astype(np.float64)) for s in range(2))
        S.set_fields(q)
        E_ref = dg.dg_energy(S.ctx)
        dq = torch.from_numpy(q).to(S.device)
        torch.cuda.synchronize(S.device)
        for _ in range(2):
            E = dg.dg_energy_static(S.ctx, dq.data_ptr())
            assert abs(E - E_or) <= tol * E_or, (E, E_or)
            assert abs(E - E_ref) <= tol * E_ref, (E, E_ref)
    finally:
        S.close()


def test_energy_static_rejects_unbound_context():
    m = I.cube_wavy_mesh(2, 2, 0.0)
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        dg.dg_set_order(ctx, 2)
        with pytest.raises(dg.DGError) as ei:
            dg.dg_energy_static(ctx, 1)
        assert ei.value.code == dg.DG_ERR_STATE
    finally:
        dg.dg_destroy(ctx)
