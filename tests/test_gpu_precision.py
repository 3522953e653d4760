"""Operator applies on the tensor cores (dg_set_op_precision): the shared
triangle mass matrix M^tri of the wedge stage's weak-form accumulation
applied with 3xTF32, TF32 or BF16 operands and FP32 accumulation, fields
FP32.  Each variant's
error against the FP64 oracle per right-hand side and after 1000 LSRK45
steps, and the discrete energy over those steps (upwind: non-increasing)."""
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

# relative L2 bars: per right-hand side of a random state, after 1000 steps
# of the smooth standing mode
# (measured on a GB300: TF32 3.3e-4 / 4.4e-4, BF16 2.8e-3 / 1.3e-2, 3xTF32 2.5e-7 / 1.4e-6)
BARS = {"fp32": (1e-5, 1e-4), "tf32x3": (1e-5, 1e-4), "tf32": (1e-3, 2e-3), "bf16": (1e-2, 5e-2)}


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("ops", ["tf32x3", "tf32", "bf16"])
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_rhs_error_against_the_oracle(ops, N):
    m = I.cube_wavy_mesh(3, 3, 0.05)
    c2, rho = I.random_material(m.K, 3, 1.0, 3.0, 0.5, 2.0)
    O = Oracle(m.VX, m.EToV, m.etype, N, c2, rho)
    q = I.random_fields(O.conn.total_nodes, 5)
    S = Solver(m.VX, m.EToV, m.etype, N, c2, rho, precision="f32", ops=ops)
    try:
        r = S.rhs(q.astype(np.float32)).cpu().numpy()
    finally:
        S.close()
    assert _rel(r, O.rhs(q)) <= BARS[ops][0]


@pytest.mark.parametrize("ops", ["tf32x3", "tf32", "bf16"])
def test_rhs_on_a_hybrid_mesh(ops):
    """Wedges under tets (the tet stage keeps FP32 CUDA-core applies)."""
    m = I.hybrid_mesh(3, 2, 1)
    c2, rho = I.random_material(m.K, 6, 1.0, 3.0, 0.5, 2.0)
    O = Oracle(m.VX, m.EToV, m.etype, 3, c2, rho)
    q = I.random_fields(O.conn.total_nodes, 2)
    S = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f32", ops=ops, bc="dirichlet", flux="central")
    O = Oracle(m.VX, m.EToV, m.etype, 3, c2, rho, bc="dirichlet", flux="central")
    try:
        r = S.rhs(q.astype(np.float32)).cpu().numpy()
    finally:
        S.close()
    assert _rel(r, O.rhs(q)) <= BARS[ops][0]


@pytest.mark.parametrize("ops", ["tf32x3", "tf32", "bf16"])
def test_1000_steps_error_and_energy(ops):
    m = I.cube_wavy_mesh(4, 4, 0.03)
    c2, rho = I.layered_wavespeed(m, (2.0, 1.5, 1.0, 1.0))
    O = Oracle(m.VX, m.EToV, m.etype, 3, c2, rho)
    q0 = I.standing_mode_unit_cube(O.conn.xyz, 0.0)
    dt = O.stable_dt(0.5)
    S = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f32", ops=ops)
    try:
        S.set_fields(q0.astype(np.float32))
        E = [S.energy()]
        for _ in range(10):
            S.step(dt, 100)
            E.append(S.energy())
        q = S.get_fields()
    finally:
        S.close()
    assert _rel(q, O.step(q0, dt, 1000)) <= BARS[ops][1]
    assert np.all(np.diff(E) <= 0.0), np.diff(E) / E[0]
