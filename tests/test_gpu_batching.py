"""Batched forms on the GPU: several shots of one mesh in one launch, and several
uneven meshes merged into one launch.  Each shot (each mesh) must reproduce the
result of its own one-shot (one-mesh) context bit for bit: the kernels do the
same arithmetic per element whatever block an element lands in."""
import numpy as np
import pytest

from oracle.dg import Solver as Oracle
from paper_1607_03399_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_1607_03399_gb300.dg import Solver  # noqa: E402


@pytest.mark.parametrize("precision", ["f32", "f64"])
@pytest.mark.parametrize("meshname", ["wedges", "hybrid"])
@pytest.mark.parametrize("order", ["outer", "inner"])
def test_shots_match_single_shot_runs(precision, meshname, order):
    m = I.cube_wavy_mesh(4, 3, 0.03) if meshname == "wedges" else I.hybrid_mesh(3, 2, 1)
    c2, rho = I.random_material(m.K, 7, 1.0, 2.0, 0.5, 1.5)
    S = 3
    pos = [(0.31, 0.62, 0.4), (0.7, 0.2, 0.55), (0.5, 0.5, 0.2)]
    shot_sources = [(s, *pos[s], 6.0 + s, 0.05, 1.0 + s) for s in range(S)]
    B = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision=precision, shots=S, shot_sources=shot_sources,
               sources=[(0.45, 0.4, 0.5, 5.0, 0.0, 0.3)], shot_order=order)
    rng = np.random.default_rng(1)
    q = rng.uniform(-1, 1, size=(S, 4, B.total_nodes)).astype(B.np_dtype)
    B.set_fields(q)
    dt = B.stable_dt(0.4)
    B.step(dt, 12)
    qb = B.get_fields()
    rb = B.rhs(q).cpu().numpy()
    B.close()
    for s in range(S):
        A = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision=precision,
                   sources=[(0.45, 0.4, 0.5, 5.0, 0.0, 0.3), (*pos[s], 6.0 + s, 0.05, 1.0 + s)])
        A.set_fields(q[s])
        A.step(dt, 12)
        assert np.array_equal(A.get_fields(), qb[s]), s
        assert np.array_equal(A.rhs(q[s]).cpu().numpy(), rb[s]), s
        A.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("order", ["outer", "inner", 2])
def test_shots_match_the_oracle_per_shot(precision, tol, order):
    """Four shots of a hybrid mesh in one launch per stage, each with its own
    Ricker source and initial state, against the oracle run shot by shot."""
    m = I.hybrid_mesh(3, 2, 1)
    c2, rho = I.random_material(m.K, 8, 1.0, 2.0, 0.5, 1.5)
    S = 4
    pos = [(0.31, 0.62, 0.4), (0.7, 0.2, 0.55), (0.5, 0.5, 0.2), (0.2, 0.8, 0.9)]
    shot_sources = [(s, *pos[s], 6.0 + s, 0.05, 1.0 + s) for s in range(S)]
    B = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision=precision, shots=S, shot_sources=shot_sources,
               shot_order=order)
    rng = np.random.default_rng(4)
    q = rng.uniform(-1, 1, size=(S, 4, B.total_nodes))
    B.set_fields(q.astype(B.np_dtype))
    dt = B.stable_dt(0.4)
    B.step(dt, 10)
    qb = B.get_fields()
    B.close()
    for s in range(S):
        O = Oracle(m.VX, m.EToV, m.etype, 3, c2, rho)
        O.add_source(*pos[s], 6.0 + s, 0.05, 1.0 + s)
        ref = O.step(q[s].astype(B.np_dtype).astype(np.float64), dt, 10)
        err = np.linalg.norm(qb[s] - ref) / np.linalg.norm(ref)
        assert err <= tol, (s, err)


def test_merged_meshes_match_separate_runs():
    """Three meshes of uneven size (wedge-only, hybrid, one-wedge) in one launch."""
    parts = [I.cube_wavy_mesh(3, 2, 0.02), I.hybrid_mesh(2, 1, 1), I.cube_wavy_mesh(1, 1, 0.0)]
    m = I.merge_meshes(parts)
    c2, rho = I.random_material(m.K, 9, 1.0, 3.0)
    Bm = Solver(m.VX, m.EToV, m.etype, 2, c2, rho, precision="f32")
    rng = np.random.default_rng(3)
    q = rng.uniform(-1, 1, size=(4, Bm.total_nodes)).astype(np.float32)
    Bm.set_fields(q)
    dt = Bm.stable_dt(0.4)
    Bm.step(dt, 8)
    qm = Bm.get_fields()
    Bm.close()
    node0 = 0
    for i, p in enumerate(parts):
        o = m.meta["offsets"][i]
        A = Solver(p.VX, p.EToV, p.etype, 2, c2[o:o + p.K], rho[o:o + p.K], precision="f32")
        n = A.total_nodes
        A.set_fields(q[:, node0:node0 + n])
        A.step(dt, 8)
        assert np.array_equal(A.get_fields(), qm[:, node0:node0 + n]), i
        A.close()
        node0 += n


@pytest.mark.parametrize("group", [2, 4])
def test_shot_groups_are_bitwise_the_shot_major_run(group):
    """Eight shots in groups of 2 or 4 (a block holds 16 or 8 elements of 2 or
    4 shots each): every shot's state after 10 steps equals the shot-major
    layout's bit for bit."""
    m = I.cube_wavy_mesh(4, 4, 0.03)
    c2, rho = I.random_material(m.K, 3, 1.0, 2.0, 0.5, 1.5)
    S = 8
    src = [(s, 0.2 + 0.08 * s, 0.5, 0.5, 6.0, 0.05, 1.0) for s in range(S)]
    q = np.random.default_rng(2).uniform(-1, 1, size=(S, 4, 0))
    out = {}
    for order in ("outer", group):
        B = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f32", shots=S, shot_sources=src, shot_order=order)
        if q.shape[2] == 0:
            q = np.random.default_rng(2).uniform(-1, 1, size=(S, 4, B.total_nodes)).astype(np.float32)
        B.set_fields(q)
        dt = B.stable_dt(0.4)
        B.step(dt, 10)
        out[order] = B.get_fields()
        B.close()
    assert np.array_equal(out["outer"], out[group])


def test_layout_autotuner_keeps_the_operator():
    """dg_autotune_layout picks a shots-per-group layout among 1, 2, 4, 8; the
    steps taken afterwards match the oracle shot by shot."""
    m = I.hybrid_mesh(3, 2, 1)
    c2, rho = I.random_material(m.K, 4, 1.0, 2.0, 0.5, 1.5)
    S = 8
    B = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f64", shots=S)
    g, us = B.autotune_layout(3)
    assert g in (1, 2, 4, 8) and us > 0
    q = np.random.default_rng(9).uniform(-1, 1, size=(S, 4, B.total_nodes))
    B.set_fields(q)
    dt = B.stable_dt(0.4)
    B.step(dt, 4)
    qb = B.get_fields()
    B.close()
    O = Oracle(m.VX, m.EToV, m.etype, 3, c2, rho)
    for s in (0, 5):
        ref = O.step(q[s], dt, 4)
        assert np.linalg.norm(qb[s] - ref) <= 1e-12 * np.linalg.norm(ref)
