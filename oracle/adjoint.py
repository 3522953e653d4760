"""Oracle misfit, its gradient by reverse-mode differentiation of LSRK45, and by
finite differences.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Misfit of pressure receivers: J(m) = 1/2 sum_{n=1..nsteps} sum_r
(l_r . p(t_n) - d_{r,n})^2, with l_r the Lagrange basis of the element holding
receiver r evaluated there.  The state follows q_n = Phi(q_{n-1}) with
Carpenter-Kennedy LSRK45 (oracle.dg.lsrk45), stage right-hand sides
r_s = A(m) Q_{s-1} + f(m, t_{n-1} + c_s dt), including the point sources.

`gradient_reverse` differentiates that recursion in reverse order with the
dense transpose of A (no structure of A is used): per step, for s = 5..1,
  lam_K += b_s lam_Q;  g += dt lam_K . dr_s/dm;  lam_Q += dt A^T lam_K;  lam_K *= a_s,
then lam_Q += R^T residual_{n-1}; dr_s/dm by central differences of the
oracle's stage right-hand side in each material parameter.  `gradient_fd`
differences J itself.  m = (kappa, rho) per element.
"""
from __future__ import annotations

import numpy as np

from . import reference as R
from .dg import Solver, WEDGE


def receiver_vector(S: Solver, x):
    """(element, l(x)) for the lowest-id element holding x."""
    for k in range(S.K):
        X = S.reference_coords(k, x)
        if S._inside(k, X):
            ref = S.W if S.conn.etype[k] == WEDGE else S.T
            return k, ref.eval(np.asarray(X)[None, :])[0]
    raise ValueError("receiver outside the mesh")


class Setup:
    def __init__(self, mesh, N, kappa, rho, sources, receivers, dt, nsteps, bc="rigid", flux="upwind"):
        self.mesh, self.N, self.sources, self.receivers = mesh, N, list(sources), list(receivers)
        self.kappa, self.rho = np.asarray(kappa, float), np.asarray(rho, float)
        self.dt, self.nsteps, self.bc, self.flux = dt, nsteps, bc, flux

    def solver(self, kappa=None, rho=None, with_sources=True) -> Solver:
        kappa = self.kappa if kappa is None else kappa
        rho = self.rho if rho is None else rho
        m = self.mesh
        S = Solver(m.VX, m.EToV, m.etype, self.N, kappa / rho, rho, bc=self.bc, flux=self.flux)
        if with_sources:
            for sc in self.sources:
                S.add_source(*sc)
        return S


def _sample_matrix(S: Solver, receivers):
    n = S.conn.total_nodes
    Rm = np.zeros((len(receivers), 4 * n))
    for i, x in enumerate(receivers):
        k, ell = receiver_vector(S, x)
        Rm[i, S.conn.offset[k]:S.conn.offset[k + 1]] = ell   # pressure rows come first in the flattening
    return Rm


def traces(st: Setup, kappa=None, rho=None):
    S = st.solver(kappa, rho)
    Rm = _sample_matrix(S, st.receivers)
    q = np.zeros((4, S.conn.total_nodes))
    out = []
    for n in range(st.nsteps):
        q = S.step(q, st.dt, 1, t0=n * st.dt)
        out.append(Rm @ q.ravel())
    return np.array(out)


def misfit(st: Setup, data, kappa=None, rho=None) -> float:
    r = traces(st, kappa, rho) - data
    return 0.5 * float((r * r).sum())


def gradient_fd(st: Setup, data, elems, h=1e-6):
    """Central differences of J in kappa_k and rho_k (relative step h)."""
    gk, gr = {}, {}
    for k in elems:
        for which, g in (("kappa", gk), ("rho", gr)):
            base = getattr(st, which)
            d = h * base[k]
            vals = []
            for sgn in (1, -1):
                m = base.copy()
                m[k] += sgn * d
                args = {"kappa": st.kappa, "rho": st.rho}
                args[which] = m
                vals.append(misfit(st, data, **args))
            g[k] = (vals[0] - vals[1]) / (2 * d)
    return gk, gr


def gradient_reverse(st: Setup, data, h=1e-6):
    """dJ/dkappa, dJ/drho for every element by reverse-mode differentiation."""
    S = st.solver()
    n = S.conn.total_nodes
    Rm = _sample_matrix(S, st.receivers)
    A = st.solver(with_sources=False).dense_A()
    # forward, keeping every stage input
    q = np.zeros((4, n))
    stages, resid = [], []
    for step in range(st.nsteps):
        t = step * st.dt
        res = np.zeros_like(q)
        Qs = []
        for s in range(5):
            Qs.append(q.copy())
            res = R.LSRK45_A[s] * res + st.dt * S.rhs(q, t + R.LSRK45_C[s] * st.dt)
            q = q + R.LSRK45_B[s] * res
        stages.append(Qs)
        resid.append(Rm @ q.ravel() - data[step])
    # stage right-hand sides of perturbed materials
    pert = []
    for k in range(S.K):
        for which in ("kappa", "rho"):
            base = getattr(st, which)
            d = h * base[k]
            pair = []
            for sgn in (1, -1):
                m = base.copy()
                m[k] += sgn * d
                args = {"kappa": st.kappa, "rho": st.rho}
                args[which] = m
                pair.append(st.solver(**args))
            pert.append((k, which, d, pair))
    gk, gr = np.zeros(S.K), np.zeros(S.K)
    lam_q = Rm.T @ resid[-1]
    for step in range(st.nsteps - 1, -1, -1):
        t = step * st.dt
        lam_k = np.zeros(4 * n)
        for s in range(4, -1, -1):
            lam_k = lam_k + R.LSRK45_B[s] * lam_q
            Q = stages[step][s]
            ts = t + R.LSRK45_C[s] * st.dt
            for (k, which, d, (Sp, Sm)) in pert:
                dr = (Sp.rhs(Q, ts) - Sm.rhs(Q, ts)).ravel() / (2 * d)
                (gk if which == "kappa" else gr)[k] += st.dt * lam_k @ dr
            lam_q = lam_q + st.dt * (A.T @ lam_k)
            lam_k = R.LSRK45_A[s] * lam_k
        if step > 0:
            lam_q = lam_q + Rm.T @ resid[step - 1]
    return gk, gr
