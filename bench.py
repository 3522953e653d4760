"""Throughput benchmark: GDOF-updates/s per LSRK45 stage of the fused wedge DG
stage on the layered-medium workload.

Workload (one GPU): [0,1]^3 footprint of 2x128x128 triangles extruded
through 16 layers with seeded Gaussian-bump interfaces (amplitude 0.2 of a
layer) = 524288 vertically mapped wedges, layered wavespeed c = 2.5, 2.0,
1.5, 1.0 by depth quartile, rho = 1, rigid walls, upwind flux, a Ricker
point source (f0 = 10, t0 = 0.1) at the domain centre, FP32 state and
arithmetic, synthetic seeded state.  N = 3 is the headline; N = 4 is
measured too.  A step is one LSRK45 step (5 stages, one fused wedge kernel
each, replayed from a CUDA graph); value = 4 * nodes * 5 * steps / time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank advances its own replica (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "layered_wedges_2x128x128x16_N3"
METRIC = "GDOF-updates/s per RK stage (wedge N=3)"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


WORKLOADS = {"full": (128, 16), "medium": (96, 16), "small": (32, 16)}


def _traffic_per_launch(mass):
    """DRAM bytes per wedge-stage launch from the committed ncu summary, or None
    when the kernel source or the mass mode differ from those of the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "wedge_stage_n3_layered524k_dram.md")
    src = os.path.join(ROOT, "paper_1607_03399_gb300", "csrc", "kernels.cuh")
    try:
        text = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    fields = dict(line.split(":", 1) for line in text.splitlines()
                  if line.startswith(("traffic_bytes", "kernel_source", "mass_mode")))
    if fields.get("kernel_source_sha256_16", "").strip() != sha or fields.get("mass_mode", "").strip() != mass:
        return None
    return int(fields["traffic_bytes_per_launch"].strip())


def _mesh(ntri=128, nlayers=16, order="column"):
    """The layered workload mesh in column-major element order (the generator's:
    each 32-element block holds two whole 16-layer columns), or the same mesh
    layer by layer (`--element-order layer`, the comparison for the column
    order's in-block vertical traces)."""
    from paper_1607_03399_gb300 import inputs as I
    m = I.bumpy_layered_mesh(ntri, nlayers)
    c2, rho = I.layered_wavespeed(m)
    if order == "layer":
        m, perm = I.layer_major(m, nlayers)
        c2, rho = c2[perm], rho[perm]
    return m, c2, rho


def _alg_bytes_per_stage(K, total_nodes, real_bytes=4):
    """The method's minimum HBM bytes for one fused stage: read q, read res,
    write res, write q (4 reals per field-DOF, 16 B in FP32) plus about 64 B
    per element of geometry, topology and material (vertex gather ~12 B
    amortised, 6 vertex ids 24 B, 5 neighbour ids 20 B, 2 material reals 8 B):
    16.40 B per field-DOF at N = 3, 16.21 B at N = 4 in FP32."""
    return 4 * real_bytes * (4 * total_nodes) + 64 * K


def _kernel_bytes_per_stage(K, nverts, total_nodes, real_bytes=4, N=3, mass="stored"):
    """What this kernel design reads and writes at least (above the method's
    minimum: its own choices): the state as above; per wedge 12 vertex
    coordinates, 5 neighbour ids and 5 orientation codes (int32) and 3
    material reals; in the stored mode the mass factor (Nt (Nt + 1) / 2
    reals), otherwise the 6 vertex ids and 3 coordinates per vertex the
    in-stage factorisation gathers."""
    dof = 4 * total_nodes
    nt = (N + 1) * (N + 2) // 2
    per_wedge = 10 * 4 + (12 + 3) * real_bytes
    if mass == "stored":
        return 4 * real_bytes * dof + K * (per_wedge + nt * (nt + 1) // 2 * real_bytes)
    return 4 * real_bytes * dof + K * (per_wedge + 6 * 4) + nverts * 3 * real_bytes


def _flops_per_wedge(N, mass="stored"):
    """Arithmetic of one wedge in one stage as the stage kernel performs it
    (an FMA counts 2), per slice j of the N + 1 slices: D_t on 4 fields
    (8 Nt Nq), the t-part and triangle-lift assembly (28 Nt), M^tri on 4
    vectors (8 Nt^2), the two triangular solves with 4 right-hand sides
    (8 Nt (Nt - 1) + 16 Nt), the strong D_r / D_s part (8 Nt^2 + 16 Nt), the
    three quadrilateral faces (fluxes 18 Nq, edge masses 8 Nq^2 each), the
    triangle-face fluxes (15 per node, 2 Nt / Nq nodes per slice) and the
    fused update (24 Nt); plus about 150 flops of geometry per wedge and, with
    the factor computed in the stage, the Cholesky factorisation
    (Nt^3 / 3 + 3 Nt^2 per wedge)."""
    nt, nq = (N + 1) * (N + 2) // 2, N + 1
    per_slice = (8 * nt * nq + 28 * nt + 8 * nt * nt + 8 * nt * (nt - 1) + 16 * nt + 8 * nt * nt + 16 * nt
                 + 3 * (18 * nq + 8 * nq * nq) + 15 * 2 * nt / nq + 24 * nt)
    f = nq * per_slice + 150
    if mass != "stored":
        f += nt ** 3 / 3 + 3 * nt * nt
    return f


def _fma_peaks():
    """Measured FP32 and FP64 CUDA-core FMA throughput (TFLOP/s) of this GPU."""
    from paper_1607_03399_gb300 import dg as _dg
    try:
        return {"fp32_tflops": _dg.dg_fma_peak(_dg.DG_F32), "fp64_tflops": _dg.dg_fma_peak(_dg.DG_F64),
                "how": "dg_fma_peak: independent FMA chains on every SM, one launch timed by CUDA events"}
    except Exception as e:  # pragma: no cover - reported, not fatal
        return {"fp32_tflops": None, "fp64_tflops": None, "error": str(e)}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-i", str(self.index), "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                try:
                    rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[2:]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _blas_threads():
    """BLAS / OpenMP thread count numpy would use in a fresh process."""
    try:
        from threadpoolctl import threadpool_info
        return sum(d.get("num_threads", 0) for d in threadpool_info()) or None
    except Exception:
        return None


def _cpu_baseline(kind_steps: int = 2):
    """Oracle on the host cores, on a bounded sample of the same recipe, in
    fresh processes: once restricted to one thread and once with every core
    allowed to the BLAS / OpenMP runtimes (the oracle's einsum contractions
    are numpy loops, so extra cores barely help; the figures show it)."""
    code = f"""
import sys, time, json, os
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle.dg import Solver
from paper_1607_03399_gb300 import inputs as I
m = I.bumpy_layered_mesh(16, 16)
c2, rho = I.layered_wavespeed(m)
S = Solver(m.VX, m.EToV, m.etype, 3, c2, rho)
q = I.random_fields(S.conn.total_nodes, 1)
dt = S.stable_dt(0.5)
q = S.step(q, dt, 1)
t = time.perf_counter()
q = S.step(q, dt, {kind_steps})
el = time.perf_counter() - t
try:
    from threadpoolctl import threadpool_info
    blas = sum(d.get("num_threads", 0) for d in threadpool_info())
except Exception:
    blas = None
print(json.dumps({{"dof": 4 * S.conn.total_nodes, "K": S.K, "sec": el, "steps": {kind_steps}, "blas_threads": blas}}))
"""
    ncpu = os.cpu_count() or 1
    runs = {}
    for label, nth in (("one_core", 1), ("all_cores", ncpu)):
        env = dict(os.environ, OMP_NUM_THREADS=str(nth), OPENBLAS_NUM_THREADS=str(nth), MKL_NUM_THREADS=str(nth))
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        runs[label] = {"value": d["dof"] * 5 * d["steps"] / d["sec"] / 1e9, "threads": nth,
                       "blas_threads": d.get("blas_threads"), "sec": d["sec"]}
    d1 = runs["one_core"]
    return {"value": d1["value"], "unit": "GDOF-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{kind_steps} LSRK45 steps (5 stages each) of the FP64 NumPy oracle on 8192 wedges "
                      f"(2x16x16 footprint x 16 bumpy layers, same recipe), N=3",
            "os_cpu_count": ncpu, "one_core": d1, "all_cores": runs["all_cores"]}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, one right-hand side +
    update (one stage) per step on a bounded sample of the workload."""
    if rank != 0:
        return
    # sample size: about a minute of oracle work for the whole run
    nside = 8 if args.steps <= 1000 else (4 if args.steps <= 4000 else 2)
    code = f"""
import sys, time, json
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle.dg import Solver
from paper_1607_03399_gb300 import inputs as I
from oracle import reference as R
m = I.bumpy_layered_mesh({nside}, 16)
c2, rho = I.layered_wavespeed(m)
S = Solver(m.VX, m.EToV, m.etype, 3, c2, rho)
q = I.random_fields(S.conn.total_nodes, 1)
res = np.zeros_like(q)
dt = S.stable_dt(0.5)
def stage(q, res, s):
    res = R.LSRK45_A[s] * res + dt * S.rhs(q)
    return q + R.LSRK45_B[s] * res, res
for i in range({args.warmup}):
    q, res = stage(q, res, i % 5)
t = time.perf_counter()
for i in range({args.steps}):
    q, res = stage(q, res, i % 5)
el = time.perf_counter() - t
print(json.dumps({{"dof": 4 * S.conn.total_nodes, "K": S.K, "sec": el}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=3000)
    d = json.loads(r.stdout.strip().splitlines()[-1])
    v = d["dof"] * args.steps / d["sec"] / 1e9
    sample = (f"one LSRK45 stage per step of the FP64 NumPy oracle on {d['K']} wedges "
              f"(2x{nside}x{nside} footprint x 16 bumpy layers, same recipe), N=3")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GDOF-updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * d["sec"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "order": 3, "sample_wedges": d["K"]},
            "cpu_baseline": {"value": v, "unit": "GDOF-updates/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "GDOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_order(N, args, torch, dev, m, c2, rho, mass, barrier=None):
    """Time args.steps LSRK45 steps after args.warmup untimed ones with CUDA
    events on the solver's stream, bracketed by a device synchronisation and
    (several ranks) a barrier on both sides."""
    from paper_1607_03399_gb300.dg import Solver
    S = Solver(m.VX, m.EToV, m.etype, N, c2, rho, precision="f32", device=str(dev),
               sources=[(0.5, 0.5, 0.5, 10.0, 0.1, 1.0)], mass=mass, ops=args.ops)
    q = np.random.default_rng(1).uniform(-1, 1, size=(4, S.total_nodes)).astype(np.float32)
    S.set_fields(q)
    dt = S.stable_dt(0.5)
    S.step(dt, args.warmup)
    S.sync()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(dev.index or 0) as clk:
        torch.cuda.synchronize(dev)
        if barrier:
            barrier()
        start.record(S.stream)
        S.step(dt, args.steps)
        end.record(S.stream)
        end.synchronize()
        torch.cuda.synchronize(dev)
        if barrier:
            barrier()
    S.sync()
    ms = start.elapsed_time(end)
    dof = 4 * S.total_nodes
    tune = None
    if not args.no_autotune:
        bpc, onthefly, split, us = S.autotune(10)
        tune = {"blocks_per_cta": bpc, "factor_in_stage": onthefly, "field_pair_split": split, "stage_us": us}
    res = {"ms": ms, "dof": dof, "clocks": clk.summary(), "solver": S, "dt": dt, "q": q, "autotune": tune}
    return res


def measure_hybrid(args, torch, dev, tet_layers=4):
    """Hybrid wedge + tet workload: 2x96x96 footprint, 12 bumpy wedge layers under
    4 flat layers of prisms split into 3 tets each (221184 tets; tet_layers=6
    gives the 331776-tet variant), N=3, FP32, c^2 from c ~ U[1,3]
    per element, rho = 1, Gaussian pressure pulse (width 0.05) at the centre,
    rigid walls, upwind.  The whole stage is timed by graph replay of LSRK45 steps,
    each element type's stage kernel separately by dg_stage_times."""
    from paper_1607_03399_gb300 import inputs as I
    from paper_1607_03399_gb300.dg import Solver
    m = I.hybrid_mesh(96, 12, tet_layers)
    c2, rho = I.random_material(m.K, 3, 1.0, 3.0)
    S = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f32", device=str(dev))
    q = I.gaussian_pulse(S.node_coords(), (0.5, 0.5, 0.5), 0.05).astype(np.float32)
    S.set_fields(q)
    dt = S.stable_dt(0.5)
    S.step(dt, args.warmup)
    S.sync()
    nsteps = max(5, args.steps // 2)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    start.record(S.stream)
    S.step(dt, nsteps)
    end.record(S.stream)
    end.synchronize()
    ms = start.elapsed_time(end)
    tw, tt = S.stage_times(20)
    Kw, Kt = int((m.etype == 6).sum()), int((m.etype == 4).sum())
    dof_w, dof_t = 4 * 40 * Kw, 4 * 20 * Kt
    st = ms / 1e3 / (5 * nsteps)
    S.close()
    peak, _ = _peaks()
    # tet algorithmic bytes: 16 B per field-DOF, per tet 4 vertex ids, 4 neighbour ids and codes, 3 material reals
    tet_bytes = 16 * dof_t + Kt * (4 * 4 + 8 * 4 + 3 * 4)
    return {"workload": f"hybrid_2x96x96_12wedge_{tet_layers}tet_layers_N3", "wedges": Kw, "tets": Kt,
            "field_dof": dof_w + dof_t, "steps": nsteps, "stage_us": st * 1e6,
            "value": (dof_w + dof_t) / st / 1e9, "unit": "GDOF-updates/s",
            "wedge_stage_us": tw, "wedge_gdofs": dof_w / (tw * 1e-6) / 1e9,
            "tet_stage_us": tt, "tet_gdofs": dof_t / (tt * 1e-6) / 1e9,
            "tet_alg_bytes": tet_bytes, "tet_frac": tet_bytes / (tt * 1e-6) / 1e9 / peak}


def measure_config1(args, torch, dev):
    """The FP64 accuracy case: 128-wedge wavy unit cube (4x4 squares split into
    32 right triangles, 4 layers, interfaces z_k = k/4 + 0.03 sin 2 pi x
    sin 2 pi y), N=3, c = rho = 1, rigid walls, upwind, the standing mode
    p = cos(pi x) cos(pi y) cos(pi z) as initial data, 200 LSRK45 steps at
    CFL 0.5.  Reports the energy every 20 steps and the final L2 error against
    the exact solution's nodal interpolant, measured in the scheme's exact mass
    norm: with c = rho = 1 the discrete energy of the difference state is half
    its squared L2 norm, so ||e|| = sqrt(2 E(q - q_exact)) through
    dg_energy_static (full state, and pressure only)."""
    from paper_1607_03399_gb300 import dg as _dg
    from paper_1607_03399_gb300 import inputs as I
    from paper_1607_03399_gb300.dg import Solver
    m = I.cube_wavy_mesh(4, 4, 0.03)
    S = Solver(m.VX, m.EToV, m.etype, 3, precision="f64", device=str(dev))
    xyz = S.node_coords()
    q0 = I.standing_mode_unit_cube(xyz, 0.0)
    dt = S.stable_dt(0.5)
    S.set_fields(q0)
    hist = [S.energy()]
    for _ in range(10):
        S.step(dt, 20)
        hist.append(S.energy())
    q = S.get_fields()
    T = S.time()
    d = q - I.standing_mode_unit_cube(xyz, T)
    dd = torch.from_numpy(np.ascontiguousarray(d)).to(dev)
    dp = dd.clone()
    dp[1:] = 0
    torch.cuda.synchronize(dev)
    err = np.sqrt(2.0 * _dg.dg_energy_static(S.ctx, dd.data_ptr()))
    err_p = np.sqrt(2.0 * _dg.dg_energy_static(S.ctx, dp.data_ptr()))
    S.close()
    return {"workload": "wavy_cube_4x4x4_128wedges_N3_fp64_standing_mode", "steps": 200, "dt": dt, "t_final": T,
            "l2_error": float(err), "l2_error_p": float(err_p),
            "energy_every_20_steps": hist, "energy_non_increasing": bool(np.all(np.diff(hist) <= 1e-14 * hist[0]))}


def measure_multishot(args, torch, dev):
    """Batched shots: 2x64x64 footprint x 32 bumpy layers = 262144 wedges, N=3,
    FP32, layered wavespeed, 64 shots each with its own Ricker source (f0 = 8)
    at a seeded position just below the surface, all advanced by one launch per
    stage, in both shot orders (shot-major blocks, and shot-inner blocks where a
    block holds 32 shots of one element); against the same 64 shots advanced one
    context launch sequence per shot (the per-shot form).  Unit: shot-steps/s."""
    from paper_1607_03399_gb300 import inputs as I
    from paper_1607_03399_gb300.dg import Solver
    S = 64
    m = I.bumpy_layered_mesh(64, 32)
    c2, rho = I.layered_wavespeed(m)
    pos = I.surface_shots(S, 4)
    n = max(3, min(args.steps // 20, 10))
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def batched(order):
        B = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f32", device=str(dev), shots=S,
                   shot_sources=[(s, *pos[s], 8.0, 0.125, 1.0) for s in range(S)], shot_order=order)
        B.set_fields(np.zeros((S, 4, B.total_nodes), dtype=np.float32))
        dt = B.stable_dt(0.5)
        B.step(dt, args.warmup)
        B.sync()
        start.record(B.stream)
        B.step(dt, n)
        end.record(B.stream)
        end.synchronize()
        B.close()
        return start.elapsed_time(end), dt

    ms_b, dt = batched("outer")
    ms_i, _ = batched("inner")
    # the layout autotuner's pick among 1, 2, 4, ..., 64 shots per group
    T = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f32", device=str(dev), shots=S,
               shot_sources=[(s, *pos[s], 8.0, 0.125, 1.0) for s in range(S)], shot_order="outer")
    g_best, us_best = T.autotune_layout(10)
    T.set_fields(np.zeros((S, 4, T.total_nodes), dtype=np.float32))
    T.step(dt, args.warmup)
    T.sync()
    start.record(T.stream)
    T.step(dt, n)
    end.record(T.stream)
    end.synchronize()
    ms_t = start.elapsed_time(end)
    T.close()
    A = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f32", device=str(dev),
               sources=[(*pos[0], 8.0, 0.125, 1.0)])
    A.set_fields(np.zeros((4, A.total_nodes), dtype=np.float32))
    A.step(dt, args.warmup)
    A.sync()
    start.record(A.stream)
    for _ in range(S):
        A.step(dt, n)
    end.record(A.stream)
    end.synchronize()
    ms_a = start.elapsed_time(end)
    A.close()
    return {"workload": "multishot_2x64x64x32_N3_64shots", "wedges": m.K, "shots": S, "steps": n,
            "batched_shot_steps_per_s": S * n / (ms_b / 1e3), "per_shot_shot_steps_per_s": S * n / (ms_a / 1e3),
            "ratio": ms_a / ms_b, "batched_gdofs": S * 4 * 40 * m.K * 5 * n / (ms_b / 1e3) / 1e9,
            "shot_inner": {"batched_shot_steps_per_s": S * n / (ms_i / 1e3), "ratio": ms_a / ms_i,
                           "batched_gdofs": S * 4 * 40 * m.K * 5 * n / (ms_i / 1e3) / 1e9},
            "autotuned": {"shots_per_group": g_best, "tuner_stage_us": us_best,
                          "batched_shot_steps_per_s": S * n / (ms_t / 1e3), "ratio": ms_a / ms_t,
                          "batched_gdofs": S * 4 * 40 * m.K * 5 * n / (ms_t / 1e3) / 1e9}}


def measure_precision(args, torch, dev):
    """Operator-precision variants (dg_set_op_precision) on the batched
    workload: 2x64x64 footprint x 32 bumpy layers = 262144 wedges, N=3, FP32
    fields, 64 shots with their Ricker sources, one launch per stage.  Every
    variant starts from the same seeded random state (drawn on the device),
    takes the warm-up and then the timed steps; reported per variant: field
    GDOF-updates/s, shot-steps/s and the relative L2 deviation of its final
    state from the FP32 CUDA-core variant's (GPU against GPU: the variants'
    errors against the FP64 oracle are measured by the precision tests)."""
    from paper_1607_03399_gb300 import inputs as I
    from paper_1607_03399_gb300.dg import Solver
    S = 64
    m = I.bumpy_layered_mesh(64, 32)
    c2, rho = I.layered_wavespeed(m)
    pos = I.surface_shots(S, 4)
    n = max(3, min(args.steps // 20, 10))
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gen = torch.Generator(device=dev)
    ref, ref_norm, out = None, None, {}
    for ops in ("fp32", "tf32x3", "tf32", "bf16"):
        B = Solver(m.VX, m.EToV, m.etype, 3, c2, rho, precision="f32", device=str(dev), shots=S,
                   shot_sources=[(s, *pos[s], 8.0, 0.125, 1.0) for s in range(S)], ops=ops)
        gen.manual_seed(4)
        q = torch.rand((S, 4, B.total_nodes), device=dev, dtype=torch.float32, generator=gen).mul_(2.0).sub_(1.0)
        B.set_fields(q)
        B.sync()
        del q
        dt = B.stable_dt(0.5)
        B.step(dt, args.warmup)
        B.sync()
        start.record(B.stream)
        B.step(dt, n)
        end.record(B.stream)
        end.synchronize()
        ms = start.elapsed_time(end)
        qf = B.get_fields(device=True)
        B.close()
        if ref is None:
            ref, ref_norm, dev_rel = qf, float(torch.linalg.vector_norm(qf, dtype=torch.float64)), 0.0
        else:
            dev_rel = float(torch.linalg.vector_norm(qf - ref, dtype=torch.float64)) / ref_norm
            del qf
        out[ops] = {"gdofs": S * 4 * 40 * m.K * 5 * n / (ms / 1e3) / 1e9, "shot_steps_per_s": S * n / (ms / 1e3),
                    "stage_us": ms * 1e3 / (5 * n), "rel_dev_from_fp32": dev_rel}
    del ref
    torch.cuda.empty_cache()
    return {"workload": "multishot_2x64x64x32_N3_64shots_random_state", "wedges": m.K, "shots": S,
            "steps": n + args.warmup, "timed_steps": n, "variants": out}


def measure_multimesh(args, torch, dev):
    """48 independent layered meshes of uneven size (footprints 2x8x8 .. 2x40x40,
    4..20 layers, seeded) merged into one context and advanced by one launch per
    stage; against 48 contexts advanced one after another.  N=3, FP32."""
    from paper_1607_03399_gb300 import inputs as I
    from paper_1607_03399_gb300.dg import Solver
    rng = np.random.default_rng(48)
    parts = [I.bumpy_layered_mesh(int(rng.integers(4, 21)) * 2, int(rng.integers(4, 21)), seed0=5000 + 50 * i)
             for i in range(48)]
    mm = I.merge_meshes(parts)
    B = Solver(mm.VX, mm.EToV, mm.etype, 3, precision="f32", device=str(dev))
    B.set_fields(np.zeros((4, B.total_nodes), dtype=np.float32))
    dt = B.stable_dt(0.5)
    n = max(5, min(args.steps // 4, 40))
    B.step(dt, args.warmup)
    B.sync()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(B.stream)
    B.step(dt, n)
    end.record(B.stream)
    end.synchronize()
    ms_b = start.elapsed_time(end)
    Ktot = mm.K
    B.close()
    solvers = [Solver(p.VX, p.EToV, p.etype, 3, precision="f32", device=str(dev)) for p in parts]
    st = torch.cuda.Stream(dev)
    for A in solvers:
        A.set_fields(np.zeros((4, A.total_nodes), dtype=np.float32))
        A.step(dt, args.warmup)
        A.sync()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for A in solvers:
        A.step(dt, n)
    for A in solvers:
        A.sync()
    s_a = time.perf_counter() - t0
    for A in solvers:
        A.close()
    return {"workload": "multimesh_48_layered_2x8x8_to_2x40x40_N3", "meshes": 48, "wedges": Ktot, "steps": n,
            "batched_mesh_steps_per_s": 48 * n / (ms_b / 1e3), "separate_mesh_steps_per_s": 48 * n / s_a,
            "ratio": s_a / (ms_b / 1e3)}


ADJOINT_SIZES = {"full": (48, 24, 8, 800), "small": (24, 12, 2, 50)}


def measure_adjoint(args, torch, dev):
    """Differentiation workload: 2x48x48 footprint x 24 layers = 110592 wedges,
    N=3, FP32 fields, two-layer c^2 with a Gaussian inclusion, 8 shots (Ricker
    f0 = 8 below the surface) and 256 surface receivers, 800 steps; misfit
    against traces of the model with a 10% stronger inclusion; checkpoints
    every 50 steps.
    Times the forward pass (with receiver sampling and checkpoints) and the
    adjoint sweep (segment re-runs, per-step stage recomputation, adjoint
    stages, gradient terms), then both again with checkpoints every 25 steps
    and stage records (the segment re-run stores the stages, no per-step
    recomputation; the forward pass records the last segment); reports the
    ratios (faster of two passes each), the peak device memory of each and
    whether the two gradients agree bit for bit; then stage records with the
    segment re-runs on a second solver, one segment ahead and concurrent with
    the reverse steps (12-step segments, two record buffers).  The headline
    ratio is the better of the two stage-record schedules.
    `--adjoint-size small` (2x24x24 x 12 layers, 2 shots, 50 steps) is the
    profiling case."""
    from paper_1607_03399_gb300 import inputs as I
    from paper_1607_03399_gb300 import adjoint as AD
    side, layers, nshots, nsteps = ADJOINT_SIZES[args.adjoint_size]
    torch.cuda.empty_cache()  # the earlier workloads' cached blocks
    m = I.bumpy_layered_mesh(side, layers)
    pos = I.surface_shots(nshots, 5)
    recs = I.surface_receivers(16)
    pb = AD.Problem(m.VX, m.EToV, m.etype, 3, 0.0, nsteps, recs, shots=nshots, checkpoint_every=50,
                    shot_sources=[(s, *pos[s], 8.0, 0.125, 1.0) for s in range(nshots)], device=str(dev))
    c2t, rho = I.inclusion_model(m, amp=0.55)
    c2, _ = I.inclusion_model(m, amp=0.5)
    S = pb.solver(c2t, rho)
    pb.dt = S.stable_dt(0.5)
    data, _ = AD.forward(S, pb)
    S.close()
    torch.cuda.synchronize(dev)
    torch.cuda.reset_peak_memory_stats(dev)
    S = pb.solver(c2, rho)

    def sweep(reps=2, R=None):
        """Faster of `reps` forward passes and of `reps` reverse sweeps (the
        host drives both step by step, so one stalled host thread shows up as
        a slow pass), the gradient, and the peak device memory."""
        _, ck = AD.forward(S, pb)  # untimed: graph capture, first allocations
        del ck
        S.sync()
        torch.cuda.synchronize(dev)
        torch.cuda.reset_peak_memory_stats(dev)
        tf, ta = [], []
        for _ in range(reps):
            t0 = time.perf_counter()
            traces, ck = AD.forward(S, pb)
            J = AD.misfit(traces, data)
            t1 = time.perf_counter()
            gk, gr = AD.reverse(S, pb, traces, data, ck, R=R)
            t2 = time.perf_counter()
            tf.append(t1 - t0)
            ta.append(t2 - t1)
            del traces, ck
        return min(tf), min(ta), J, gk, gr, torch.cuda.max_memory_allocated(dev)

    f1, a1, J, gk, gr, peak = sweep()
    # the same gradient from stage records: checkpoints every 25 steps, ten
    # fields per step of the segment, no per-step recomputation, the last
    # segment recorded by the forward pass
    pb.checkpoint_every, pb.stage_records = 25, True
    f2, a2, J2, gk2, gr2, peak2 = sweep()
    # the same with the segment re-runs on a second solver, concurrent with the
    # reverse steps (two record buffers: 12-step segments)
    torch.cuda.empty_cache()
    R = pb.solver(c2, rho)
    pb.checkpoint_every = 12
    f3, a3, J3, gk3, gr3, peak3 = sweep(R=R)
    R.close()
    S.close()
    best = min(a2 / f2, a3 / f3)
    return {"workload": f"adjoint_2x{side}x{side}x{layers}_N3_{nshots}shots_{len(recs)}rec", "wedges": m.K,
            "shots": nshots, "receivers": len(recs), "steps": nsteps,
            "adjoint_over_forward": best, "misfit": J, "timing": "faster of 2 passes each",
            "stage_records_overlapped": {"checkpoint_every": 12, "forward_s": f3, "adjoint_s": a3,
                                         "adjoint_over_forward": a3 / f3, "peak_device_gb": peak3 / 1e9,
                                         "same_gradient": bool(J3 == J and np.array_equal(gk, gk3)
                                                               and np.array_equal(gr, gr3))},
            "gradient_norm": float(np.sqrt((gk ** 2).sum() + (gr ** 2).sum())),
            "recompute": {"checkpoint_every": 50, "forward_s": f1, "adjoint_s": a1,
                          "adjoint_over_forward": a1 / f1, "peak_device_gb": peak / 1e9},
            "stage_records": {"checkpoint_every": 25, "forward_s": f2, "adjoint_s": a2,
                              "adjoint_over_forward": a2 / f2, "peak_device_gb": peak2 / 1e9,
                              "same_gradient": bool(J2 == J and np.array_equal(gk, gk2) and np.array_equal(gr, gr2))}}


def _max_over_ranks(x, dist, dev):
    """The largest of the ranks' values of x (the slowest rank times the job);
    x itself with one process.  Works with the gloo and the NCCL backends."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _gdofs(dof, stages, seconds, world):
    """Whole-job GDOF-updates/s: every rank advances its own replica of `dof`
    field DOF through `stages` Runge-Kutta stages in `seconds` (the slowest
    rank's time)."""
    return dof * stages / seconds / 1e9 * world


def measure_adjoint_hybrid(args, torch, dev):
    """Differentiation on a hybrid mesh: 2x48x48 footprint, 8 bumpy wedge layers
    under 4 layers of tets (36864 wedges + 55296 tets), N=3, FP32, the two-layer
    model with its inclusion, 4 shots, 256 receivers just below the surface (in
    the tets), 200 steps, stage records in 25-step segments.  Reverse over
    forward time (faster of two passes each), and the gradient against the
    recomputing schedule bit for bit."""
    from paper_1607_03399_gb300 import inputs as I
    from paper_1607_03399_gb300 import adjoint as AD
    m = I.hybrid_mesh(48, 8, 4)
    nshots, nsteps = 4, 200
    pos = I.surface_shots(nshots, 5)
    recs = I.surface_receivers(16)
    pb = AD.Problem(m.VX, m.EToV, m.etype, 3, 0.0, nsteps, recs, shots=nshots, checkpoint_every=25,
                    stage_records=True, shot_sources=[(s, *pos[s], 8.0, 0.125, 1.0) for s in range(nshots)],
                    device=str(dev))
    c2t, rho = I.inclusion_model(m, amp=0.55)
    c2, _ = I.inclusion_model(m, amp=0.5)
    S = pb.solver(c2t, rho)
    pb.dt = S.stable_dt(0.5)
    data, _ = AD.forward(S, pb)
    S.close()
    S = pb.solver(c2, rho)
    _, ck = AD.forward(S, pb)  # untimed: graph capture, first allocations
    del ck
    tf, ta = [], []
    for _ in range(2):
        t0 = time.perf_counter()
        traces, ck = AD.forward(S, pb)
        t1 = time.perf_counter()
        gk, gr = AD.reverse(S, pb, traces, data, ck)
        t2 = time.perf_counter()
        tf.append(t1 - t0)
        ta.append(t2 - t1)
        del traces, ck
    pb.stage_records, pb.checkpoint_every = False, 50
    traces, ck = AD.forward(S, pb)
    gk2, gr2 = AD.reverse(S, pb, traces, data, ck)
    S.close()
    return {"workload": f"adjoint_hybrid_2x48x48_8wedge_4tet_layers_N3_{nshots}shots_{len(recs)}rec",
            "wedges": int((m.etype == 6).sum()), "tets": int((m.etype == 4).sum()), "shots": nshots,
            "steps": nsteps, "checkpoint_every": 25, "forward_s": min(tf), "adjoint_s": min(ta),
            "adjoint_over_forward": min(ta) / min(tf), "timing": "faster of 2 passes each",
            "same_gradient_as_recompute": bool(np.array_equal(gk, gk2) and np.array_equal(gr, gr2)),
            "gradient_norm": float(np.sqrt((gk ** 2).sum() + (gr ** 2).sum()))}


def run_ours(args, rank, world):
    import torch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    ntri, nlay = WORKLOADS[args.workload]
    m, c2, rho = _mesh(ntri, nlay, args.element_order)
    orders = [int(x) for x in args.orders.split(",")]
    out = {}
    barrier = dist.barrier if world > 1 else None
    for N in orders:
        r = measure_order(N, args, torch, dev, m, c2, rho, args.mass, barrier)
        r["ms_max"] = _max_over_ranks(r["ms"], dist, dev)
        out[N] = r
        if N == orders[0] and not args.no_e2e:
            S = r["solver"]
            # end to end through the public API with host buffers: per step
            # upload the state from pinned memory, one LSRK45 step, download
            qh = torch.from_numpy(r["q"]).pin_memory()
            qo = torch.empty_like(qh).pin_memory()
            ne = max(3, min(args.steps, 20))
            S.set_fields(qh.numpy())
            torch.cuda.synchronize(dev)
            if barrier:
                barrier()
            t0 = time.perf_counter()
            for _ in range(ne):
                S.set_fields(qh.numpy())
                S.step(r["dt"], 1)
                from paper_1607_03399_gb300 import dg as _dg
                _dg.dg_get_fields(S.ctx, qo.data_ptr(), 0)
            e2e_s = _max_over_ranks((time.perf_counter() - t0) / ne, dist, dev)
            r["e2e"] = {"value": _gdofs(r["dof"], 5, e2e_s, world), "unit": "GDOF-updates/s",
                        "h2d_bytes_per_step": int(qh.numel() * 4), "d2h_bytes_per_step": int(qo.numel() * 4)}
        r["solver"].close()
        r["solver"] = None
    hybrid = measure_hybrid(args, torch, dev) if (rank == 0 and not args.no_hybrid) else None
    hybrid6 = measure_hybrid(args, torch, dev, tet_layers=6) if (rank == 0 and not args.no_hybrid) else None
    config1 = measure_config1(args, torch, dev) if (rank == 0 and not args.no_config1) else None
    multishot = measure_multishot(args, torch, dev) if (rank == 0 and not args.no_batched) else None
    multimesh = measure_multimesh(args, torch, dev) if (rank == 0 and not args.no_batched) else None
    precision = measure_precision(args, torch, dev) if (rank == 0 and not args.no_batched) else None
    adjoint = measure_adjoint(args, torch, dev) if (rank == 0 and not args.no_adjoint) else None
    adjoint_hybrid = measure_adjoint_hybrid(args, torch, dev) if (rank == 0 and not args.no_adjoint) else None
    # the headline order once more with the other way of applying the mass inverse
    other = {"stored": "onthefly", "onthefly": "stored"}[args.mass]
    alt = None
    if not args.no_alt:
        alt = measure_order(orders[0], args, torch, dev, m, c2, rho, other, barrier)
        alt["ms_max"] = _max_over_ranks(alt["ms"], dist, dev)
        alt["solver"].close()
        alt["solver"] = None
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peak, peak_kind = _peaks()
    fma = _fma_peaks()
    fp32_peak = fma.get("fp32_tflops")
    r3 = out[orders[0]]
    K, nverts = m.K, m.VX.shape[0]
    ms_step = r3["ms_max"] / args.steps
    value = _gdofs(r3["dof"], 5 * args.steps, r3["ms_max"] / 1e3, world)
    stage_s = r3["ms"] / 1e3 / (5 * args.steps)
    alg = _alg_bytes_per_stage(K, r3["dof"] // 4)
    kbytes = _kernel_bytes_per_stage(K, nverts, r3["dof"] // 4, N=orders[0], mass=args.mass)
    achieved = alg / stage_s / 1e9

    def flop_rate(N, mode, st):
        tf = _flops_per_wedge(N, mode) * K / st / 1e12
        return {"tflops": tf, "fp32_peak_tflops": fp32_peak, "frac_fp32": tf / fp32_peak if fp32_peak else None,
                "flops_per_field_dof": _flops_per_wedge(N, mode) / (4 * (N + 1) ** 2 * (N + 2) / 2)}

    by_order = {}
    for N, r in out.items():
        st = r["ms"] / 1e3 / (5 * args.steps)
        a = _alg_bytes_per_stage(K, r["dof"] // 4)
        kb = _kernel_bytes_per_stage(K, nverts, r["dof"] // 4, N=N, mass=args.mass)
        by_order[str(N)] = {"autotune": r["autotune"],
                            "value": _gdofs(r["dof"], 5 * args.steps, r["ms_max"] / 1e3, world),
                            "ms_per_step": r["ms_max"] / args.steps, "stage_us": st * 1e6,
                            "alg_bytes_per_stage": a, "achieved_gbs": a / st / 1e9,
                            "frac": a / st / 1e9 / peak, "kernel_bytes_per_stage": kb,
                            "kernel_bytes_frac": kb / st / 1e9 / peak, "dof": r["dof"],
                            "alu": flop_rate(N, args.mass, st)}
    by_mass = {}
    if alt is not None:
        for mode, r in ((args.mass, r3), (other, alt)):
            st = r["ms"] / 1e3 / (5 * args.steps)
            a = _alg_bytes_per_stage(K, r["dof"] // 4)
            kb = _kernel_bytes_per_stage(K, nverts, r["dof"] // 4, N=orders[0], mass=mode)
            by_mass[mode] = {"value": _gdofs(r["dof"], 5 * args.steps, r["ms_max"] / 1e3, world), "stage_us": st * 1e6,
                             "alg_bytes_per_stage": a, "frac": a / st / 1e9 / peak,
                             "kernel_bytes_per_stage": kb, "kernel_bytes_frac": kb / st / 1e9 / peak,
                             "alu": flop_rate(orders[0], mode, st)}
    cpu = _cpu_baseline() if (world == 1 and not args.no_cpu) else None
    line = {
        "metric": METRIC, "value": value, "unit": "GDOF-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.workload == "full" else f"layered_wedges_2x{ntri}x{ntri}x{nlay}",
                   "wedges": K, "order": orders[0], "field_dof": r3["dof"], "element_order": args.element_order,
                   "l2_flush": "inputs larger than L2 (3 state buffers of %.0f MB)" % (r3["dof"] * 4 / 1e6),
                   "bc": "rigid", "flux": "upwind", "source": "Ricker f0=10 t0=0.1 at (0.5,0.5,0.5)",
                   "mass": args.mass, "ops": args.ops},
        "roofline": {"kernel": f"k_wedge_stage<{orders[0]}>", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": _traffic_per_launch(args.mass) if (args.workload == "full" and orders[0] == 3
                                                                   and args.element_order == "column") else None,
                     "alg_bytes_per_launch": alg,
                     "alg_bytes": "the method's minimum: 16 B per field-DOF (read q and res, write res and q) "
                                  "+ 64 B per wedge of mesh data",
                     "kernel_bytes_per_launch": kbytes,
                     "kernel_bytes": "what this kernel must move: the state as above, 100 B of mesh tables per "
                                     "wedge and the stored mass factor (overhead above the method's minimum)",
                     "alu": by_order[str(orders[0])]["alu"]},
        "fma_peaks": fma,
        "config1": config1,
        "hybrid6": hybrid6,
        "by_order": by_order,
        "by_mass": by_mass or None,
        "hybrid": hybrid,
        "multishot": multishot,
        "multimesh": multimesh,
        "precision": precision,
        "adjoint": adjoint,
        "adjoint_hybrid": adjoint_hybrid,
        "e2e": r3.get("e2e"),
        "gpu_launches": 6 * args.steps,  # per step: 5 stage launches and one clock launch
        "clocks": r3["clocks"],
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="full", choices=sorted(WORKLOADS))
    ap.add_argument("--orders", default="3,4", help="orders to measure; the first is the headline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--mass", default="stored", choices=["stored", "onthefly"],
                    help="how the stage applies the wedge mass inverse (stored factor or factored in the stage)")
    ap.add_argument("--no-alt", action="store_true", help="skip the headline order in the other mass mode")
    ap.add_argument("--no-hybrid", action="store_true", help="skip the hybrid wedge + tet workload")
    ap.add_argument("--no-batched", action="store_true", help="skip the multi-shot and multi-mesh workloads")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (gradient) workload")
    ap.add_argument("--no-config1", action="store_true", help="skip the FP64 accuracy case (128 wedges, 200 steps)")
    ap.add_argument("--element-order", default="column", choices=["column", "layer"],
                    help="element order of the layered workload (layer: the comparison for the column order)")
    ap.add_argument("--adjoint-size", default="full", choices=sorted(ADJOINT_SIZES),
                    help="size of the adjoint workload (small: the profiling case)")
    ap.add_argument("--no-autotune", action="store_true", help="skip the launch-variant autotuner after timing")
    ap.add_argument("--ops", default="fp32", choices=["fp32", "tf32x3", "tf32", "bf16"],
                    help="how the wedge stage applies the shared triangle operators (CUDA-core FP32 or tensor cores)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
