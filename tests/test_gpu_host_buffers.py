"""Host field buffers: pinned, device-mapped memory is packed and unpacked by the
layout kernel directly over the CPU-GPU link, pageable memory through a bulk
copy.  Both must give the same device state and the same host result, bit for
bit, for wedges and tets, both precisions and several shots (element blocks
with padding lanes included)."""
import numpy as np
import pytest

from paper_1607_03399_gb300 import dg
from paper_1607_03399_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_1607_03399_gb300.dg import Solver  # noqa: E402


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("meshname,N", [("wedges", 3), ("hybrid", 2), ("hybrid", 4)])
def test_pinned_and_pageable_host_buffers_agree(precision, meshname, N):
    m = I.cube_wavy_mesh(3, 3, 0.04) if meshname == "wedges" else I.hybrid_mesh(3, 2, 1)
    c2, rho = I.random_material(m.K, 3, 1.0, 2.0, 0.6, 1.4)
    S = Solver(m.VX, m.EToV, m.etype, N, c2, rho, precision=precision, shots=2,
               sources=[(0.4, 0.45, 0.5, 5.0, 0.05, 1.0)])
    q = np.random.default_rng(4).uniform(-1, 1, size=S.field_shape).astype(S.np_dtype)
    dt = S.stable_dt(0.4)

    # pageable: bulk copy + layout kernel
    S.set_fields(q)
    assert np.array_equal(S.get_fields(), q)
    S.step(dt, 3)
    ref = S.get_fields()

    # pinned: the layout kernel reads and writes host memory directly
    qp = torch.from_numpy(q.copy()).pin_memory()
    out = torch.empty_like(qp).pin_memory()
    dg.dg_set_fields(S.ctx, qp.data_ptr(), 0)
    dg.dg_get_fields(S.ctx, out.data_ptr(), 0)
    assert np.array_equal(out.numpy(), q)
    dg.dg_set_fields(S.ctx, qp.data_ptr(), 0)
    S.step(dt, 3)
    dg.dg_get_fields(S.ctx, out.data_ptr(), 0)
    assert np.array_equal(out.numpy(), ref)

    # mixed: pinned in, device out, pageable in, pinned out
    dg.dg_set_fields(S.ctx, qp.data_ptr(), 0)
    assert np.array_equal(S.get_fields(device=True).cpu().numpy(), q)
    S.set_fields(q)
    dg.dg_get_fields(S.ctx, out.data_ptr(), 0)
    assert np.array_equal(out.numpy(), q)
    S.close()
