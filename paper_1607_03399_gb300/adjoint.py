"""Receiver misfit and its gradient with respect to the per-element material,
through the library's discrete adjoint of dg_step (every step of the sweep runs
in the CUDA library; this module orders the calls and keeps checkpoints).

J(c^2, rho) = 1/2 sum_{n=1..nsteps} sum_shots sum_r (p_r(t_n) - d_r(t_n))^2,
with p_r the pressure at receiver r after step n.  The forward pass keeps a
checkpoint of the state every `checkpoint_every` steps; the reverse pass
re-runs each segment from its checkpoint to recover the step states and calls
dg_adjoint_step once per step, which recomputes that step's five stages and
accumulates dJ/dkappa, dJ/drho.  With `stage_records` the segment re-run
instead stores every step's stage inputs and right-hand sides (ten fields per
step, dg_step_record_chain) and the reverse steps read them back
(dg_adjoint_step_recorded): one forward pass less per step for
checkpoint_every x 10 fields of device memory; the forward pass records the
last segment itself, so that segment is not re-run.  The gradient is the same
bit for bit.  The chain rule to (c^2, rho) uses kappa = rho c^2.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .dg import Solver


@dataclass
class Problem:
    """A seismic-style inversion setup on one mesh of wedges."""
    VX: np.ndarray
    EToV: np.ndarray
    etype: np.ndarray
    N: int
    dt: float
    nsteps: int
    receivers: list                     # [(x, y, z)]
    shot_sources: list = field(default_factory=list)   # [(shot, x, y, z, f0, t0, amp)]
    shots: int = 1
    precision: str = "f32"
    bc: str = "rigid"
    flux: str = "upwind"
    checkpoint_every: int = 50
    stage_records: bool = False
    shot_order: str = "outer"
    device: str = "cuda:0"

    def solver(self, c2, rho) -> Solver:
        return Solver(self.VX, self.EToV, self.etype, self.N, np.asarray(c2, dtype=np.float64),
                      np.asarray(rho, dtype=np.float64), bc=self.bc, flux=self.flux, precision=self.precision,
                      device=self.device, shots=self.shots, shot_sources=self.shot_sources,
                      receivers=self.receivers, shot_order=self.shot_order)


@dataclass
class Checkpoints:
    """What the forward pass keeps for the reverse pass: the state and the
    solver's own time at every checkpoint step (accumulated step by step, so a
    re-run from a checkpoint evaluates the sources at exactly the forward
    pass's stage times) and, with stage records, the records of the last
    segment (steps records_from .. nsteps - 1), which the reverse pass then
    does not re-run."""
    states: dict
    records: list | None = None
    records_from: int = -1


def forward(S: Solver, pb: Problem, q0=None):
    """Traces [nsteps][shots][receivers] (device tensor) and the Checkpoints."""
    torch = S.torch
    S.set_fields(np.zeros(S.field_shape, dtype=S.np_dtype) if q0 is None else q0)
    traces = torch.empty((pb.nsteps, pb.shots, S.nrec), dtype=S.dtype, device=S.device)
    C = pb.checkpoint_every
    ck = Checkpoints({0: (S.save_state(), S.time())})
    if pb.stage_records and pb.nsteps > 0:
        ck.records_from = ((pb.nsteps - 1) // C) * C
        ck.records = [S.new_record() for _ in range(pb.nsteps - ck.records_from)]
    for n in range(1, pb.nsteps + 1):
        if ck.records is not None and n - 1 >= ck.records_from:
            S.step_record(pb.dt, ck.records[n - 1 - ck.records_from])
        else:
            S.step(pb.dt, 1)
        S.sample(traces[n - 1])
        if n % C == 0 and n < pb.nsteps:
            ck.states[n] = (S.save_state(), S.time())
    S.sync()
    return traces, ck


def misfit(traces, data) -> float:
    r = traces.double() - data.double()
    return 0.5 * float((r * r).sum())


def reverse(S: Solver, pb: Problem, traces, data, ck, R: Solver | None = None):
    """dJ/dkappa, dJ/drho per element after a forward() on the same solver.

    With stage records and a second solver R of the same problem (same mesh,
    material, options and shots, its own state and stream), the segment
    re-runs run on R, one segment ahead, concurrently with the reverse steps
    on S: two record buffers alternate, and CUDA events order each buffer's
    re-run before its reverse steps and its reverse steps before its next
    re-run.  The gradient is the same bit for bit."""
    torch = S.torch
    resid = (traces - data.to(traces.dtype)).contiguous()
    if getattr(S, "d_adj", None) is None:
        S.adjoint_bind()
    else:
        S.adjoint_reset()
    C = pb.checkpoint_every
    starts = list(range(0, pb.nsteps, C))
    if pb.stage_records and R is not None:
        order = list(reversed(starts))
        own = ck.records if (ck.records is not None and order[0] == ck.records_from) else None
        first = own if own is not None else []
        bufs = [first + [S.new_record() for _ in range(min(C, pb.nsteps) - len(first))],
                [S.new_record() for _ in range(min(C, pb.nsteps))]]
        free = [None, None]  # per buffer: event after its last reverse step

        def rerun(i):
            """Re-run segment order[i] on R into buffer i % 2; the event that marks it done."""
            s0 = order[i]
            s1 = min(s0 + C, pb.nsteps)
            b = i % 2
            if free[b] is not None:
                R.stream.wait_event(free[b])
            R.load_state(*ck.states[s0])
            R.step_record_chain(pb.dt, bufs[b][:s1 - s0])
            ev = torch.cuda.Event()
            ev.record(R.stream)
            return ev

        ready = None if own is not None else rerun(0)
        for i, s0 in enumerate(order):
            s1 = min(s0 + C, pb.nsteps)
            b = i % 2
            nxt = rerun(i + 1) if i + 1 < len(order) else None
            if ready is not None:
                S.stream.wait_event(ready)
            for n in range(s1, s0, -1):
                S.adjoint_inject(resid[n - 1])
                S.adjoint_step_recorded(pb.dt, bufs[b][n - 1 - s0])
            ev = torch.cuda.Event()
            ev.record(S.stream)
            free[b] = ev
            ready = nxt
        R.sync()
        S.sync()
        return S.adjoint_gradient()
    if pb.stage_records:
        recs = ck.records
        if recs is None or len(recs) < min(C, pb.nsteps):
            recs = (recs or []) + [S.new_record() for _ in range(min(C, pb.nsteps) - len(recs or []))]
        for s0 in reversed(starts):
            s1 = min(s0 + C, pb.nsteps)
            # records of the steps q_n -> q_{n+1}, n = s0 .. s1 - 1 (the last
            # segment's come from the forward pass)
            if not (s0 == ck.records_from and ck.records is not None):
                S.load_state(*ck.states[s0])
                S.step_record_chain(pb.dt, recs[:s1 - s0])
            for n in range(s1, s0, -1):
                S.adjoint_inject(resid[n - 1])
                S.adjoint_step_recorded(pb.dt, recs[n - 1 - s0])
        S.sync()
        return S.adjoint_gradient()
    for s0 in reversed(starts):
        s1 = min(s0 + C, pb.nsteps)
        # states q_{s0} .. q_{s1 - 1} of the segment
        S.load_state(*ck.states[s0])
        states = [ck.states[s0]]
        for n in range(s0 + 1, s1):
            S.step(pb.dt, 1)
            states.append((S.save_state(), S.time()))
        for n in range(s1, s0, -1):
            S.adjoint_inject(resid[n - 1])
            S.load_state(*states[n - 1 - s0])
            S.adjoint_step(pb.dt)
    S.sync()
    return S.adjoint_gradient()


def material_gradient(c2, rho, gk, gr):
    """(dJ/dc^2, dJ/drho at fixed c^2) from (dJ/dkappa, dJ/drho at fixed kappa)."""
    c2 = np.asarray(c2, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    return rho * gk, gr + c2 * gk


def misfit_and_gradient(pb: Problem, c2, rho, data):
    S = pb.solver(c2, rho)
    try:
        traces, ck = forward(S, pb)
        J = misfit(traces, data)
        gk, gr = reverse(S, pb, traces, data, ck)
    finally:
        S.close()
    return J, *material_gradient(c2, rho, gk, gr)


def _autograd_function():
    import torch

    class AcousticMisfit(torch.autograd.Function):
        """J(c^2, rho) with dJ/dc^2 and dJ/drho from the discrete adjoint.  The
        forward pass runs the wave simulation and keeps its checkpoints; the
        backward pass runs the adjoint sweep."""

        @staticmethod
        def forward(ctx, c2, rho, pb, data):
            S = pb.solver(c2.detach().cpu().numpy(), rho.detach().cpu().numpy())
            traces, ck = forward(S, pb)
            J = torch.tensor(misfit(traces, data), dtype=torch.float64)
            if not any(ctx.needs_input_grad[:2]):
                # no gradient will be asked for: release the solver and its
                # checkpoints now instead of holding device memory with the graph
                S.close()
                ctx.state = None
                return J
            # (dropping the graph without backward frees them too: the solver
            # closes itself when the last reference goes)
            ctx.state = (S, pb, traces, data, ck)
            ctx.save_for_backward(c2, rho)
            return J

        @staticmethod
        def backward(ctx, gJ):
            c2, rho = ctx.saved_tensors
            S, pb, traces, data, ck = ctx.state
            try:
                gk, gr = reverse(S, pb, traces, data, ck)
            finally:
                S.close()
                ctx.state = None
            g2, grho = material_gradient(c2.detach().cpu().numpy(), rho.detach().cpu().numpy(), gk, gr)
            s = float(gJ)
            return (torch.as_tensor(s * g2, dtype=c2.dtype, device=c2.device),
                    torch.as_tensor(s * grho, dtype=rho.dtype, device=rho.device), None, None)

    return AcousticMisfit


def acoustic_misfit(c2, rho, pb: Problem, data):
    """Differentiable J(c^2, rho) (torch tensors of per-element values)."""
    return _autograd_function().apply(c2, rho, pb, data)
