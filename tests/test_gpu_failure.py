"""Failure detection without a GPU fault: a kernel whose bounded device-side
wait cannot complete (an mbarrier armed for bytes no copy delivers) runs its
wait out, reports DG_ERR_TIMEOUT through the device error word and returns;
the host sees the status at the next synchronising call, the word is cleared,
and the context keeps working (steps still match the oracle)."""
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


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_expired_wait_reports_timeout_and_context_survives(precision, tol):
    m = I.hybrid_mesh(2, 2, 1)
    c2, rho = I.random_material(m.K, 4, 1.0, 2.0, 0.5, 1.5)
    S = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision=precision)
    O = Oracle(m.VX, m.EToV, m.etype, 3, c2, rho)
    try:
        q = I.random_fields(S.total_nodes, 3)
        S.set_fields(q.astype(S.np_dtype))
        dg.dg_sync(S.ctx)
        dg.dg_expire_wait(S.ctx)
        with pytest.raises(dg.DGError) as ei:
            dg.dg_sync(S.ctx)
        assert ei.value.code == dg.DG_ERR_TIMEOUT
        # the error word was cleared by the report; the state is untouched
        dg.dg_sync(S.ctx)
        assert np.array_equal(S.get_fields(), q.astype(S.np_dtype))
        # a timeout raised between steps surfaces at the energy call too
        dg.dg_expire_wait(S.ctx)
        with pytest.raises(dg.DGError) as ei:
            dg.dg_energy(S.ctx)
        assert ei.value.code == dg.DG_ERR_TIMEOUT
        # and the context still steps correctly
        dt = O.stable_dt(0.4)
        S.step(dt, 3)
        dg.dg_sync(S.ctx)
        ref = O.step(q, dt, 3)
        assert np.linalg.norm(S.get_fields() - ref) <= tol * np.linalg.norm(ref)
    finally:
        S.close()


def test_expire_wait_needs_a_bound_context():
    m = I.cube_wavy_mesh(2, 2, 0.0)
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        dg.dg_set_order(ctx, 2)
        with pytest.raises(dg.DGError) as ei:
            dg.dg_expire_wait(ctx)
        assert ei.value.code == dg.DG_ERR_STATE
    finally:
        dg.dg_destroy(ctx)
