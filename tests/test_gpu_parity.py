"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (relative L2 over all fields and nodes): FP64 1e-12; FP32 1e-5 per
right-hand side and 1e-4 after 1000 LSRK45 steps.  Meshes span several
32-element blocks with ragged tails, wedge-only, tet-only and hybrid cases,
both boundary conditions and both fluxes; the throughput workload (524288
wedges, N = 3 and 4) and the hybrid workload (221184 wedges + 221184 tets)
are checked on sampled elements against oracle patches."""
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

from patch_util import face_adjacency, node_index, patch, submesh  # noqa: E402

MESHES = {
    # 128 wedges (4 blocks), the FP64 test configuration
    "wavy128": lambda: I.cube_wavy_mesh(4, 4, 0.03),
    # 150 wedges: ragged last block
    "bumpy150": lambda: I.layered_wedge_mesh(5, 5, 3, lambda k, x, y: k / 3 + (0.05 * np.sin(3 * x) * np.cos(2 * y) if 0 < k < 3 else 0)),
    # 2x3x3 tri columns: 18 wedge + 54 tets (hybrid, ragged)
    "hybrid": lambda: I.hybrid_mesh(3, 2, 1),
    # tets only
    "tets": lambda: I.tet_box_mesh(2, 2),
    # one wedge
    "single": lambda: I.cube_wavy_mesh(1, 1, 0.0),
}


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / np.linalg.norm(b))


def _pair(mesh, N, precision, bc="rigid", flux="upwind", seed=3, mass="stored"):
    c2, rho = I.random_material(mesh.K, seed, 1.0, 3.0, 0.5, 2.0)
    S = Solver(mesh.VX, mesh.EToV, mesh.etype, N, c2, rho, bc=bc, flux=flux, precision=precision, mass=mass)
    O = Oracle(mesh.VX, mesh.EToV, mesh.etype, N, c2, rho, bc=bc, flux=flux)
    return S, O


@pytest.mark.parametrize("meshname", list(MESHES))
@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("bc,flux", [("rigid", "upwind"), ("dirichlet", "central")])
@pytest.mark.parametrize("mass", ["stored", "onthefly"])
def test_rhs_parity_f64(meshname, N, bc, flux, mass):
    S, O = _pair(MESHES[meshname](), N, "f64", bc, flux, mass=mass)
    q = I.random_fields(S.total_nodes, 11)
    err = _rel(S.rhs(q).cpu().numpy(), O.rhs(q))
    S.close()
    assert err <= 1e-12, err


@pytest.mark.parametrize("meshname", list(MESHES))
@pytest.mark.parametrize("N", [1, 2, 3, 4])
@pytest.mark.parametrize("bc,flux", [("rigid", "upwind"), ("dirichlet", "upwind"), ("rigid", "central")])
@pytest.mark.parametrize("mass", ["stored", "onthefly"])
def test_rhs_parity_f32(meshname, N, bc, flux, mass):
    S, O = _pair(MESHES[meshname](), N, "f32", bc, flux, mass=mass)
    q = I.random_fields(S.total_nodes, 12).astype(np.float32)
    err = _rel(S.rhs(q).cpu().numpy(), O.rhs(q.astype(np.float64)))
    S.close()
    assert err <= 1e-5, err


@pytest.mark.parametrize("mass", ["stored", "onthefly"])
def test_config1_fp64_200_steps(mass):
    """128-wedge wavy unit cube, N=3, rigid walls, upwind, standing mode,
    200 LSRK45 steps at CFL 0.5: state within 1e-12 of the oracle, energy
    within 1e-12 and non-increasing, L2 error to the exact solution small."""
    m = I.cube_wavy_mesh(4, 4, 0.03)
    S = Solver(m.VX, m.EToV, m.etype, 3, precision="f64", mass=mass)
    O = Oracle(m.VX, m.EToV, m.etype, 3)
    q0 = I.standing_mode_unit_cube(O.conn.xyz, 0.0)
    dt = O.stable_dt(0.5)
    assert abs(S.stable_dt(0.5) - dt) < 1e-15 * dt
    S.set_fields(q0)
    q_ref = q0.copy()
    E_gpu = [S.energy()]
    for _ in range(10):
        S.step(dt, 20)
        q_ref = O.step(q_ref, dt, 20)
        E_gpu.append(S.energy())
    q = S.get_fields()
    assert _rel(q, q_ref) <= 1e-12
    assert abs(E_gpu[-1] - O.energy(q_ref)) <= 1e-12 * E_gpu[0]
    assert np.all(np.diff(E_gpu) <= 1e-14 * E_gpu[0])
    assert abs(S.time() - 200 * dt) < 1e-12
    err = O.l2_error(q, I.standing_mode_unit_cube, 200 * dt)
    assert np.sqrt((err ** 2).sum()) < 1e-3
    S.close()


def test_fp32_1000_steps():
    """FP32 state after 1000 LSRK45 steps within 1e-4 of the FP64 oracle."""
    m = I.cube_wavy_mesh(4, 4, 0.03)
    c2, rho = I.layered_wavespeed(m, (2.0, 1.5, 1.0, 1.0))
    S = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f32")
    O = Oracle(m.VX, m.EToV, m.etype, 3, c2, rho)
    q0 = I.standing_mode_unit_cube(O.conn.xyz, 0.0)
    dt = O.stable_dt(0.5)
    S.set_fields(q0)
    S.step(dt, 1000)
    q_ref = O.step(q0, dt, 1000)
    err = _rel(S.get_fields(), q_ref)
    S.close()
    assert err <= 1e-4, err


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-6)])
@pytest.mark.parametrize("meshname", ["wavy128", "hybrid"])
def test_energy(precision, tol, meshname):
    S, O = _pair(MESHES[meshname](), 3, precision)
    q = I.random_fields(S.total_nodes, 5)
    S.set_fields(q)
    qq = S.get_fields().astype(np.float64)
    E = S.energy()
    S.close()
    assert abs(E - O.energy(qq)) <= tol * E


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_fields_roundtrip_and_rhs_in_place(precision):
    S, O = _pair(MESHES["hybrid"](), 2, precision)
    q = I.random_fields(S.total_nodes, 8).astype(S.np_dtype)
    S.set_fields(q)
    assert np.array_equal(S.get_fields(), q)                 # pack/unpack is exact
    dq = torch.from_numpy(q).cuda()
    ref = S.rhs(dq).cpu().numpy()
    dg.dg_rhs(S.ctx, dq.data_ptr(), dq.data_ptr())           # in place
    S.sync()
    assert np.array_equal(dq.cpu().numpy(), ref)
    assert np.array_equal(S.get_fields(), q)                 # state untouched by dg_rhs
    S.close()


def test_nonfinite_state_reported():
    S, _ = _pair(MESHES["wavy128"](), 2, "f32")
    q = I.random_fields(S.total_nodes, 1).astype(np.float32)
    q[2, 17] = np.nan
    S.set_fields(q)
    with pytest.raises(dg.DGError) as ei:
        S.energy()
    assert ei.value.code == dg.DG_ERR_NONFINITE
    q[2, 17] = 0.0
    S.set_fields(q)
    assert np.isfinite(S.energy())
    S.close()


def test_two_contexts_interleaved():
    """Contexts of different order and precision on one device keep their own
    operator tables."""
    A, OA = _pair(MESHES["wavy128"](), 3, "f32")
    B, OB = _pair(MESHES["hybrid"](), 2, "f64")
    qa = I.random_fields(A.total_nodes, 1).astype(np.float32)
    qb = I.random_fields(B.total_nodes, 2)
    for _ in range(2):
        assert _rel(A.rhs(qa).cpu().numpy(), OA.rhs(qa.astype(np.float64))) <= 1e-5
        assert _rel(B.rhs(qb).cpu().numpy(), OB.rhs(qb)) <= 1e-12
    A.close()
    B.close()


@pytest.mark.parametrize("N,mass", [(3, "stored"), (4, "stored"), (3, "onthefly")])
def test_full_size_sampled(N, mass):
    """The 524288-wedge layered workload (2x128x128 triangles x 16 bumpy
    layers, layered wavespeed) in FP32 as the benchmark runs it: sampled
    elements of one right-hand side and of one full LSRK45 step (5 stages)
    against oracle patches of radius 1 and 5."""
    m = I.bumpy_layered_mesh(128, 16)
    c2, rho = I.layered_wavespeed(m)
    S = Solver(m.VX, m.EToV, m.etype, N, c2, rho, precision="f32", mass=mass)
    Np = (N + 1) ** 2 * (N + 2) // 2
    rng = np.random.default_rng(N)
    q = rng.uniform(-1, 1, size=(4, S.total_nodes)).astype(np.float32)
    nbr = face_adjacency(m.EToV, m.etype)
    # include the first and last block and both domain boundaries
    seeds = np.unique(np.concatenate([[0, 31, m.K - 1], rng.integers(0, m.K, 13)]))
    r_gpu = S.rhs(q).cpu().numpy()
    dt = S.stable_dt(0.5)
    S.set_fields(q)
    S.step(dt, 1)
    q1_gpu = S.get_fields()
    S.close()
    for radius, what in ((1, "rhs"), (5, "step")):
        for s in seeds:
            elems = patch(nbr, [s], radius)
            VXs, Es, ts = submesh(m.VX, m.EToV, m.etype, elems)
            O = Oracle(VXs, Es, ts, N, c2[elems], rho[elems])
            gid = node_index(np.full(m.K, Np), elems)
            qs = q[:, gid].astype(np.float64)
            loc = int(np.searchsorted(elems, s))
            sl = slice(loc * Np, (loc + 1) * Np)
            glob = slice(s * Np, (s + 1) * Np)
            if what == "rhs":
                ref = O.rhs(qs)[:, sl]
                got = r_gpu[:, glob]
            else:
                ref = O.step(qs, dt, 1)[:, sl]
                got = q1_gpu[:, glob]
            assert _rel(got, ref) <= 1e-5, (what, s)


@pytest.mark.parametrize("precision,tol,rhs_tol", [("f64", 1e-12, 1e-12), ("f32", 2e-5, 1e-5)])
def test_point_sources(precision, tol, rhs_tol):
    """Ricker point sources (one inside a wedge, one on a vertex shared by
    several elements: the lowest element id takes it, one in a tet) over 40
    LSRK45 steps from rest, and dg_rhs at the resulting simulation time."""
    m = I.hybrid_mesh(3, 2, 2)
    c2, rho = I.random_material(m.K, 2, 1.0, 3.0, 0.5, 2.0)
    srcs = [(0.41, 0.37, 0.22, 6.0, 0.05, 1.0),          # inside a wedge
            (1.0 / 3.0, 2.0 / 3.0, 0.75, 8.0, 0.08, -2.0),  # footprint vertex inside the tet layers
            (0.5, 0.5, 0.3, 5.0, 0.0, 0.5)]
    S = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision=precision, sources=srcs)
    O = Oracle(m.VX, m.EToV, m.etype, 3, c2, rho)
    for sc in srcs:
        O.add_source(*sc)
    dt = O.stable_dt(0.4)
    q0 = np.zeros((4, S.total_nodes))
    S.set_fields(q0)
    S.step(dt, 40)
    q_ref = O.step(q0, dt, 40)
    q = S.get_fields()
    assert np.linalg.norm(q_ref) > 0
    assert _rel(q, q_ref) <= tol
    r_ref = O.rhs(q_ref, 40 * dt)
    r = S.rhs(q_ref.astype(S.np_dtype)).cpu().numpy()
    assert _rel(r, r_ref) <= rhs_tol
    S.close()


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_stage_times_leave_the_state_alone(precision):
    """dg_stage_times times both element types and changes neither the state
    nor the next step (hybrid mesh, both precisions)."""
    S, O = _pair(MESHES["hybrid"](), 3, precision)
    q = I.random_fields(S.total_nodes, 4).astype(np.float32)
    S.set_fields(q)
    tw, tt = S.stage_times(3)
    assert tw > 0 and tt > 0
    assert np.array_equal(S.get_fields(), q)
    dt = O.stable_dt(0.4)
    S.step(dt, 2)
    assert _rel(S.get_fields(), O.step(q.astype(np.float64), dt, 2)) <= 1e-5
    S.close()


@pytest.mark.parametrize("N", [3, 4])
def test_autotune_keeps_the_operator(N):
    """dg_autotune picks a launch variant; steps taken with it still match the oracle."""
    S, O = _pair(MESHES["bumpy150"](), N, "f32")
    q = I.random_fields(S.total_nodes, 6).astype(np.float32)
    S.set_fields(q)
    bpc, onthefly, split, us = S.autotune(3)
    assert bpc in (1, 2) and us > 0 and not (split and onthefly)
    dt = O.stable_dt(0.4)
    S.step(dt, 3)
    assert _rel(S.get_fields(), O.step(q.astype(np.float64), dt, 3)) <= 1e-5
    S.close()


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-4)])
@pytest.mark.parametrize("N", [2, 3, 4])
def test_hybrid_steps(precision, tol, N):
    """Hybrid mesh (wedge layers under a tet layer, ragged blocks of both
    types), 20 LSRK45 steps of a Gaussian pulse: both stage kernels'
    Runge-Kutta updates against the oracle (the tet residual comes through
    shared memory in FP32 at N <= 3, from global memory otherwise)."""
    m = MESHES["hybrid"]()
    S, O = _pair(m, N, precision, seed=9)
    q0 = I.gaussian_pulse(O.conn.xyz, (0.45, 0.5, 0.6), 0.2)
    dt = O.stable_dt(0.4)
    S.set_fields(q0)
    S.step(dt, 20)
    q = S.get_fields()
    S.close()
    ref = O.step(q0, dt, 20)
    assert _rel(q, ref) <= tol


def test_full_size_hybrid_sampled():
    """The hybrid workload as the benchmark runs it (2x96x96 footprint, 12 bumpy
    wedge layers under 4 flat layers of prisms split into 3 tets, N = 3, FP32):
    sampled wedges and tets, including both sides of the wedge/tet interface,
    of one right-hand side and one LSRK45 step against oracle patches."""
    m = I.hybrid_mesh(96, 12, 4)
    c2, rho = I.random_material(m.K, 3, 1.0, 3.0)
    N = 3
    S = Solver(m.VX, m.EToV, m.etype, N, c2, rho, precision="f32")
    npe = np.where(m.etype == 6, (N + 1) ** 2 * (N + 2) // 2, (N + 1) * (N + 2) * (N + 3) // 6)
    off = np.concatenate([[0], np.cumsum(npe)])
    rng = np.random.default_rng(7)
    q = rng.uniform(-1, 1, size=(4, S.total_nodes)).astype(np.float32)
    nbr = face_adjacency(m.EToV, m.etype)
    tets = np.nonzero(m.etype == 4)[0]
    wedges = np.nonzero(m.etype == 6)[0]
    iface = tets[np.any((nbr[tets] >= 0) & (m.etype[np.maximum(nbr[tets], 0)] == 6), axis=1)]
    seeds = np.unique(np.concatenate([[0, m.K - 1, tets[0], tets[-1]], rng.choice(tets, 3), rng.choice(wedges, 2),
                                      rng.choice(iface, 3)]))
    r_gpu = S.rhs(q).cpu().numpy()
    dt = S.stable_dt(0.5)
    S.set_fields(q)
    S.step(dt, 1)
    q1_gpu = S.get_fields()
    S.close()
    for radius, what in ((1, "rhs"), (5, "step")):
        for s in seeds:
            elems = patch(nbr, [s], radius)
            VXs, Es, ts = submesh(m.VX, m.EToV, m.etype, elems)
            O = Oracle(VXs, Es, ts, N, c2[elems], rho[elems])
            gid = node_index(npe, elems)
            qs = q[:, gid].astype(np.float64)
            loc = int(np.searchsorted(elems, s))
            lo = int(npe[elems[:loc]].sum())
            sl = slice(lo, lo + int(npe[s]))
            glob = slice(int(off[s]), int(off[s + 1]))
            if what == "rhs":
                ref = O.rhs(qs)[:, sl]
                got = r_gpu[:, glob]
            else:
                ref = O.step(qs, dt, 1)[:, sl]
                got = q1_gpu[:, glob]
            assert _rel(got, ref) <= 1e-5, (what, int(s), int(m.etype[s]))


@pytest.mark.parametrize("flux", ["upwind", "central"])
def test_hybrid_energy_stability_f64(flux):
    """Energy stability on a hybrid mesh (Section 4.1; the exact Jacobian-weighted
    wedge mass inverse keeps it on the vertically mapped wedges): over 200
    LSRK45 steps the discrete energy never increases; the central flux keeps it
    to 1e-8 (only the time integrator dissipates), the upwind penalty
    dissipates.  The GPU energies equal the oracle's at every sample."""
    m = MESHES["hybrid"]()
    S, O = _pair(m, 3, "f64", flux=flux, seed=9)
    q = I.gaussian_pulse(O.conn.xyz, (0.45, 0.5, 0.6), 0.2)
    dt = O.stable_dt(0.4)
    S.set_fields(q)
    E = [S.energy()]
    for _ in range(10):
        S.step(dt, 20)
        q = O.step(q, dt, 20)
        E.append(S.energy())
        assert abs(E[-1] - O.energy(q)) <= 1e-12 * E[0]
    S.close()
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-13 * E[0])
    if flux == "central":
        assert E[-1] >= (1 - 1e-8) * E[0]
    else:
        assert E[-1] < (1 - 1e-3) * E[0]


def test_hybrid_fp32_1000_steps():
    """FP32 state on the hybrid mesh after 1000 LSRK45 steps within 1e-4 of the
    FP64 oracle (wedge and tet kernels, both Runge-Kutta update paths)."""
    m = MESHES["hybrid"]()
    S, O = _pair(m, 3, "f32", seed=9)
    q0 = I.gaussian_pulse(O.conn.xyz, (0.45, 0.5, 0.6), 0.2)
    dt = O.stable_dt(0.4)
    S.set_fields(q0)
    S.step(dt, 1000)
    q = S.get_fields()
    S.close()
    ref = O.step(q0, dt, 1000)
    assert _rel(q, ref) <= 1e-4


@pytest.mark.parametrize("N", [2, 3, 4])
@pytest.mark.parametrize("split", [1, -1])
def test_field_pair_split_stage(N, split):
    """The wedge stage split over field pairs (two threads per element and
    slice) and the one-thread form, forced either way: right-hand side and
    ten LSRK45 steps with sources on a hybrid mesh against the oracle."""
    from paper_1607_03399_gb300 import dg as _dg
    m = MESHES["hybrid"]()
    c2, rho = I.random_material(m.K, 5, 1.0, 3.0, 0.5, 2.0)
    src = (0.41, 0.37, 0.22, 6.0, 0.05, 1.0)
    S = Solver(m.VX, m.EToV, m.etype, N, c2, rho, precision="f32", sources=[src])
    O = Oracle(m.VX, m.EToV, m.etype, N, c2, rho)
    O.add_source(*src)
    _dg.dg_set_launch_variant(S.ctx, 2 + (8 if split > 0 else 0))  # one block per CTA, split or not
    q = I.random_fields(S.total_nodes, 13)
    r = S.rhs(q.astype(np.float32)).cpu().numpy()
    assert _rel(r, O.rhs(q)) <= 1e-5
    dt = O.stable_dt(0.4)
    S.set_fields(q.astype(np.float32))
    S.step(dt, 10)
    assert _rel(S.get_fields(), O.step(q.astype(np.float32).astype(np.float64), dt, 10)) <= 1e-5
    S.close()


@pytest.mark.parametrize("meshname", ["wavy128", "hybrid", "tets"])
@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_order_5(meshname, precision, tol):
    """N = 5 (Nt = 21, Np = 126 per wedge, 56 per tet): one right-hand side and
    three LSRK45 steps against the oracle (FP64 tets read their lift rows from
    global memory at this order)."""
    S, O = _pair(MESHES[meshname](), 5, precision, bc="rigid", flux="upwind", seed=4)
    q = I.random_fields(S.total_nodes, 21)
    qs = q.astype(S.np_dtype)
    err = _rel(S.rhs(qs).cpu().numpy(), O.rhs(qs.astype(np.float64)))
    assert err <= tol, err
    dt = O.stable_dt(0.4)
    S.set_fields(qs)
    S.step(dt, 3)
    err = _rel(S.get_fields(), O.step(qs.astype(np.float64), dt, 3))
    S.close()
    assert err <= tol, err


def test_order_5_refusals():
    """At N = 5 the tensor-core variants and the FP64 adjoint are refused with
    DG_ERR_ORDER instead of failing at launch."""
    from paper_1607_03399_gb300 import dg as _dg
    m = MESHES["wavy128"]()
    with pytest.raises(_dg.DGError) as ei:
        Solver(m.VX, m.EToV, m.etype, 5, precision="f32", ops="tf32")
    assert ei.value.code == _dg.DG_ERR_ORDER
    S = Solver(m.VX, m.EToV, m.etype, 5, precision="f64")
    with pytest.raises(_dg.DGError) as ei:
        S.adjoint_bind()
    assert ei.value.code == _dg.DG_ERR_ORDER
    S.close()


@pytest.mark.parametrize("mass", ["stored", "onthefly"])
def test_element_order_gives_the_same_bits(mass):
    """The same layered mesh listed column by column (every vertical neighbour
    in its 32-element block) and layer by layer (none is, so the stage takes
    the variant that requests the triangle-face neighbour nodes early): element
    by element the same bits after ten LSRK45 steps with a point source."""
    m = I.bumpy_layered_mesh(8, 8)
    ml, perm = I.layer_major(m, 8)
    c2, rho = I.random_material(m.K, 5, 1.0, 3.0, 0.8, 1.3)
    Np = 40
    src = (0.413, 0.371, 0.523, 6.0, 0.05, 1.0)
    A = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f32", sources=[src], mass=mass)
    B = Solver(ml.VX, ml.EToV, ml.etype, 3, c2[perm], rho[perm], precision="f32", sources=[src], mass=mass)
    q = I.random_fields(A.total_nodes, 7, np.float32)
    idx = (perm[:, None] * Np + np.arange(Np)).ravel()  # node j of the layer order is node idx[j]
    A.set_fields(q)
    B.set_fields(np.ascontiguousarray(q[:, idx]))
    dt = A.stable_dt(0.4)
    A.step(dt, 10)
    B.step(dt, 10)
    qa, qb = A.get_fields(), B.get_fields()
    A.close()
    B.close()
    assert np.array_equal(qa[:, idx], qb)
