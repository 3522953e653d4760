"""The discrete adjoint on the GPU (wedge and hybrid meshes): the adjoint step is the
transpose of the forward step in the energy inner product (dot test, FP64),
and the misfit gradient equals the oracle's reverse-mode gradient, central
differences of the GPU misfit, and the torch.autograd path."""
import numpy as np
import pytest

from oracle import adjoint as OA
from oracle import reference as ORef
from oracle.dg import Solver as Oracle
from paper_1607_03399_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("CUDA not available", allow_module_level=True)

from paper_1607_03399_gb300 import adjoint as AD  # noqa: E402
from paper_1607_03399_gb300.dg import Solver  # noqa: E402


@pytest.mark.parametrize("flux,bc,meshname", [("upwind", "rigid", "wedges"), ("central", "rigid", "wedges"),
                                              ("upwind", "dirichlet", "wedges"), ("upwind", "rigid", "hybrid"),
                                              ("central", "dirichlet", "hybrid")])
def test_adjoint_step_dot_product(flux, bc, meshname):
    """<Phi v, W P mu_n> = <v, W P mu_{n-1}> for one step (mu = P W^{-1} lambda)."""
    m = I.cube_wavy_mesh(3, 2, 0.05) if meshname == "wedges" else I.hybrid_mesh(2, 2, 1)
    c2, rho = I.random_material(m.K, 2, 1.0, 2.0, 0.7, 1.3)
    S = Solver(m.VX, m.EToV, m.etype, 2, c2, rho, precision="f64", flux=flux, bc=bc)
    O = Oracle(m.VX, m.EToV, m.etype, 2, c2, rho, flux=flux, bc=bc)
    n = S.total_nodes
    rng = np.random.default_rng(5)
    v = rng.standard_normal((4, n))
    mu = rng.standard_normal((4, n))
    dt = O.stable_dt(0.4)
    S.set_fields(v)
    S.step(dt, 1)
    phiv = S.get_fields()
    S.adjoint_bind()
    S.adjoint_set(mu, ORef.LSRK45_B[4] * mu)
    S.set_fields(v)
    S.adjoint_step(dt)
    mu0 = S.adjoint_get()
    S.close()
    W = O.energy_weights()
    P = np.ones(4 * n)
    P[n:] = -1.0
    lhs = phiv.ravel() @ (W @ (P * mu.ravel()))
    rhs = v.ravel() @ (W @ (P * mu0.ravel()))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _problem(precision, ck=5, meshname="wedges"):
    m = I.cube_wavy_mesh(2, 1, 0.05) if meshname == "wedges" else I.hybrid_mesh(2, 1, 1)
    rng = np.random.default_rng(0)
    kap, rho = rng.uniform(1, 2, m.K), rng.uniform(0.8, 1.3, m.K)
    src = (0.4, 0.6, 0.5, 3.0, 0.2, 1.0)
    recs = [(0.7, 0.3, 0.6), (0.2, 0.2, 0.3)]
    st = OA.Setup(m, 1, kap, rho, [src], recs, 0.02, 12)
    data = OA.traces(st) * 0.9 + 0.01
    pb = AD.Problem(m.VX, m.EToV, m.etype, 1, 0.02, 12, recs, shot_sources=[(0, *src)], precision=precision,
                    checkpoint_every=ck)
    return m, st, data, pb, kap, rho


def _gpu_gradient(pb, kap, rho, data):
    S = pb.solver(kap / rho, rho)
    d = torch.as_tensor(data[:, None, :], dtype=S.dtype, device=S.device)
    traces, ckp = AD.forward(S, pb)
    J = AD.misfit(traces, d)
    gk, gr = AD.reverse(S, pb, traces, d, ckp)
    S.close()
    return J, gk, gr


@pytest.mark.parametrize("precision,tol", [("f64", 1e-9), ("f32", 1e-5)])
@pytest.mark.parametrize("meshname", ["wedges", "hybrid"])
def test_gradient_matches_oracle_reverse_mode(precision, tol, meshname):
    m, st, data, pb, kap, rho = _problem(precision, meshname=meshname)
    J, gk, gr = _gpu_gradient(pb, kap, rho, data)
    ok, orr = OA.gradient_reverse(st, data)
    assert abs(J - OA.misfit(st, data)) <= (1e-12 if precision == "f64" else 1e-4) * abs(J)
    g = np.concatenate([gk, gr])
    go = np.concatenate([ok, orr])
    assert np.linalg.norm(g - go) <= tol * np.linalg.norm(go)


def test_gradient_matches_gpu_finite_differences():
    m, st, data, pb, kap, rho = _problem("f64", ck=4)
    J, gk, gr = _gpu_gradient(pb, kap, rho, data)
    for k in (1, 4, 6):
        for which in ("kappa", "rho"):
            base = kap if which == "kappa" else rho
            h = 1e-6 * base[k]
            vals = []
            for sgn in (1, -1):
                b = base.copy()
                b[k] += sgn * h
                kk, rr = (b, rho) if which == "kappa" else (kap, b)
                S = pb.solver(kk / rr, rr)
                tr, _ = AD.forward(S, pb)
                vals.append(AD.misfit(tr, torch.as_tensor(data[:, None, :], dtype=S.dtype, device=S.device)))
                S.close()
            fd = (vals[0] - vals[1]) / (2 * h)
            g = gk[k] if which == "kappa" else gr[k]
            assert abs(g - fd) <= 1e-6 * abs(fd), (k, which, g, fd)


def test_gradient_matches_finite_differences_on_16_random_elements():
    """FP64, N = 3, 128 deformed wedges, one Ricker source and a 3x3x3 grid of
    receivers, 30 steps: dJ/dkappa or dJ/drho (drawn at random) of 16 randomly
    drawn elements against central differences of the GPU misfit."""
    m = I.cube_wavy_mesh(4, 4, 0.03)
    assert m.K >= 100
    rng = np.random.default_rng(16)
    kap, rho = rng.uniform(1, 2, m.K), rng.uniform(0.8, 1.3, m.K)
    g1 = (0.25, 0.5, 0.75)
    recs = [(x, y, z) for x in g1 for y in g1 for z in g1]
    src = (0.4, 0.6, 0.5, 3.0, 0.0, 1.0)
    O = Oracle(m.VX, m.EToV, m.etype, 3, kap / rho, rho)
    dt = O.stable_dt(0.4)
    pb = AD.Problem(m.VX, m.EToV, m.etype, 3, dt, 30, recs, shot_sources=[(0, *src)], precision="f64",
                    checkpoint_every=10)
    S = pb.solver(kap / rho, rho)
    tr, _ = AD.forward(S, pb)
    S.close()
    data = (0.9 * tr + 0.01).clone()
    J, gk, gr = _gpu_gradient(pb, kap, rho, data.cpu().numpy()[:, 0, :])
    gmax = max(np.abs(gk).max(), np.abs(gr).max())
    elems = rng.choice(m.K, size=16, replace=False)
    which = rng.integers(0, 2, size=16)
    for k, w in zip(elems, which):
        base = kap if w == 0 else rho
        h = 1e-6 * base[k]
        vals = []
        for sgn in (1, -1):
            b = base.copy()
            b[k] += sgn * h
            kk, rr = (b, rho) if w == 0 else (kap, b)
            S = pb.solver(kk / rr, rr)
            t, _ = AD.forward(S, pb)
            vals.append(AD.misfit(t, data))
            S.close()
        fd = (vals[0] - vals[1]) / (2 * h)
        g = gk[k] if w == 0 else gr[k]
        assert abs(g - fd) <= 1e-6 * max(abs(fd), 1e-3 * gmax), (k, w, g, fd)


def test_autograd_function():
    m, st, data, pb, kap, rho = _problem("f64")
    c2 = torch.tensor(kap / rho, dtype=torch.float64, requires_grad=True)
    rh = torch.tensor(rho, dtype=torch.float64, requires_grad=True)
    d = torch.as_tensor(data[:, None, :], dtype=torch.float64, device="cuda")
    J = AD.acoustic_misfit(c2, rh, pb, d)
    J.backward()
    J2, g2, grho = AD.misfit_and_gradient(pb, kap / rho, rho, d)
    assert abs(float(J.detach()) - J2) <= 1e-12 * J2
    assert np.allclose(c2.grad.numpy(), g2, rtol=1e-10, atol=0)
    assert np.allclose(rh.grad.numpy(), grho, rtol=1e-10, atol=0)


@pytest.mark.parametrize("order,meshname", [("outer", "wedges"), ("inner", "wedges"), ("inner", "hybrid")])
def test_shots_sum_their_gradients(order, meshname):
    m = I.cube_wavy_mesh(3, 2, 0.03) if meshname == "wedges" else I.hybrid_mesh(2, 2, 1)
    c2, rho = I.random_material(m.K, 11, 1.0, 2.0, 0.8, 1.2)
    recs = [(0.2, 0.7, 0.8), (0.6, 0.4, 0.2), (0.8, 0.8, 0.5)]
    srcs = [(0, 0.3, 0.3, 0.4, 4.0, 0.25, 1.0), (1, 0.7, 0.6, 0.6, 5.0, 0.2, -0.5)]
    kw = dict(VX=m.VX, EToV=m.EToV, etype=m.etype, N=2, dt=0.01, nsteps=15, receivers=recs, precision="f64",
              checkpoint_every=6)
    rng = np.random.default_rng(2)
    data = torch.as_tensor(rng.standard_normal((15, 2, 3)) * 1e-3, dtype=torch.float64, device="cuda")
    pb2 = AD.Problem(shot_sources=srcs, shots=2, shot_order=order, **kw)
    J, g2, gr = AD.misfit_and_gradient(pb2, c2, rho, data)
    Js, g2s, grs = 0.0, 0.0, 0.0
    for s in range(2):
        pb1 = AD.Problem(shot_sources=[(0, *srcs[s][1:])], shots=1, **kw)
        j, a, b = AD.misfit_and_gradient(pb1, c2, rho, data[:, s:s + 1].contiguous())
        Js, g2s, grs = Js + j, g2s + a, grs + b
    assert abs(J - Js) <= 1e-12 * abs(J)
    assert np.allclose(g2, g2s, rtol=1e-9, atol=1e-14 * np.abs(g2).max())
    assert np.allclose(gr, grs, rtol=1e-9, atol=1e-14 * np.abs(gr).max())


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_step_record_is_the_step(precision):
    """dg_step_record advances the state and time exactly like dg_step (two
    shots with sources, so the stage times matter) and its slot 0 holds the
    packed input state of the step; dg_step_record_chain gives the same
    state and time and records that drive the adjoint identically."""
    m = I.cube_wavy_mesh(3, 2, 0.05)
    c2, rho = I.random_material(m.K, 4, 1.0, 2.0, 0.7, 1.3)
    kw = dict(precision=precision, shots=2,
              shot_sources=[(0, 0.4, 0.5, 0.5, 4.0, 0.1, 1.0), (1, 0.6, 0.4, 0.5, 5.0, 0.1, -1.0)])
    A = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, **kw)
    B = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, **kw)
    v = np.random.default_rng(8).standard_normal(A.field_shape)
    dt = A.stable_dt(0.4)
    A.set_fields(v)
    B.set_fields(v)
    A.step(dt, 3)
    recs = [B.new_record() for _ in range(3)]
    before = []
    for r in recs:
        before.append(B.save_state())
        B.step_record(dt, r)
    B.sync()
    fa, fb = A.get_fields(), B.get_fields()
    assert np.array_equal(fa, fb)
    assert A.time() == B.time()
    nb = B.field_bytes
    for r, q in zip(recs, before):
        assert torch.equal(r[:nb], q)
    # the chained form: the same records, state and time
    Cs = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, **kw)
    Cs.set_fields(v)
    chain = [Cs.new_record() for _ in range(3)]
    Cs.step_record_chain(dt, chain)
    Cs.sync()
    assert np.array_equal(Cs.get_fields(), fb)
    assert Cs.time() == B.time()
    # records are compared through their use (lanes and bytes past the packed
    # data are never written): three recorded adjoint steps from each set
    mu = np.random.default_rng(9).standard_normal(B.field_shape)
    outs = []
    for S_, rr in ((B, recs), (Cs, chain)):
        S_.adjoint_bind()
        S_.adjoint_set(mu, 0.3 * mu)
        for r in reversed(rr):
            S_.adjoint_step_recorded(dt, r)
        outs.append((S_.adjoint_get(), *S_.adjoint_gradient()))
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert np.abs(outs[0][1]).max() > 0
    A.close()
    B.close()
    Cs.close()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_stage_records_give_the_same_gradient(precision):
    """The reverse sweep from stage records equals the one that recomputes the
    stages, bit for bit (segments of 5, 5 and 2 steps)."""
    m, st, data, pb, kap, rho = _problem(precision)
    J, gk, gr = _gpu_gradient(pb, kap, rho, data)
    pb.stage_records = True
    J2, gk2, gr2 = _gpu_gradient(pb, kap, rho, data)
    assert J == J2
    assert np.abs(gk).max() > 0 and np.abs(gr).max() > 0
    assert np.array_equal(gk, gk2) and np.array_equal(gr, gr2)


def test_fp32_gradient_against_fp64_on_the_inclusion_workload():
    """The differentiation workload's recipe at reduced size (2x24x24 footprint
    x 12 layers, two-layer model with the shallow Gaussian inclusion, 2 shots,
    256 surface receivers, 200 steps): the FP32 misfit and gradient against
    the FP64 GPU run (itself pinned to the oracle's reverse mode above)."""
    m = I.bumpy_layered_mesh(24, 12)
    pos = I.surface_shots(2, 5)
    recs = I.surface_receivers(16)
    out = {}
    for prec in ("f64", "f32"):
        pb = AD.Problem(m.VX, m.EToV, m.etype, 3, 0.0, 200, recs, shots=2, checkpoint_every=50,
                        shot_sources=[(s, *pos[s], 8.0, 0.125, 1.0) for s in range(2)], precision=prec)
        c2t, rho = I.inclusion_model(m, amp=0.55)
        c2, _ = I.inclusion_model(m, amp=0.5)
        S = pb.solver(c2t, rho)
        pb.dt = S.stable_dt(0.5)
        data, _ = AD.forward(S, pb)
        S.close()
        S = pb.solver(c2, rho)
        traces, ck = AD.forward(S, pb)
        J = AD.misfit(traces, data)
        gk, gr = AD.reverse(S, pb, traces, data, ck)
        S.close()
        out[prec] = (J, np.concatenate([gk, gr]))
    (J64, g64), (J32, g32) = out["f64"], out["f32"]
    assert abs(J32 - J64) <= 1e-4 * J64
    assert np.linalg.norm(g32 - g64) <= 2e-4 * np.linalg.norm(g64)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_overlapped_reruns_give_the_same_gradient(precision):
    """Stage records with the segment re-runs on a second solver, concurrent with
    the reverse steps (three segments): the gradient equals the one-solver
    sweep's bit for bit."""
    m, st, data, pb, kap, rho = _problem(precision, ck=4)
    pb.stage_records = True
    S = pb.solver(kap / rho, rho)
    R = pb.solver(kap / rho, rho)
    d = torch.as_tensor(data[:, None, :], dtype=S.dtype, device=S.device)
    traces, ck = AD.forward(S, pb)
    gk1, gr1 = AD.reverse(S, pb, traces, d, ck)
    traces, ck = AD.forward(S, pb)
    gk2, gr2 = AD.reverse(S, pb, traces, d, ck, R=R)
    S.close()
    R.close()
    assert np.array_equal(gk1, gk2) and np.array_equal(gr1, gr2)


def test_autograd_without_gradients_releases_the_solver():
    """A forward pass whose inputs need no gradient keeps no solver."""
    m, st, data, pb, kap, rho = _problem("f64")
    c2 = torch.tensor(kap / rho, dtype=torch.float64)
    rh = torch.tensor(rho, dtype=torch.float64)
    d = torch.as_tensor(data[:, None, :], dtype=torch.float64, device="cuda")
    J = AD.acoustic_misfit(c2, rh, pb, d)
    J2, _, _ = AD.misfit_and_gradient(pb, kap / rho, rho, d)
    assert not J.requires_grad and abs(float(J) - J2) <= 1e-12 * J2
