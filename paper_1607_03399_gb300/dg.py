"""Python binding of the dgwedge C ABI (include/dgwedge.h).

Argument marshalling only: every step of the solver runs in libdgwedge.so.
The functions keep the C names; `Solver` bundles them with device buffers
allocated through PyTorch (which provides device memory and streams only).

Loading fails loudly when the shared library is missing: build it with
`python -c "import __graft_entry__ as g; g.build()"` or
`python paper_1607_03399_gb300/build.py`.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int64, c_size_t, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgwedge.so")

DG_OK = 0
DG_ERR_ARG, DG_ERR_MESH, DG_ERR_ORDER, DG_ERR_CUDA, DG_ERR_STATE, DG_ERR_TIMEOUT, DG_ERR_NONFINITE = range(-1, -8, -1)
DG_TET, DG_WEDGE = 4, 6
DG_BC_DIRICHLET, DG_BC_RIGID = 0, 1
DG_FLUX_UPWIND, DG_FLUX_CENTRAL = 0, 1
DG_F32, DG_F64 = 0, 1
DG_MASS_ONTHEFLY, DG_MASS_STORED = 0, 1
DG_SHOTS_OUTER, DG_SHOTS_INNER = 0, 1
DG_OPS_FP32, DG_OPS_TF32X3, DG_OPS_TF32, DG_OPS_BF16 = 0, 1, 2, 3

EXPORTS = ("dg_mesh_create", "dg_set_order", "dg_set_material", "dg_add_source", "dg_set_shots", "dg_add_shot_source", "dg_set_shot_order", "dg_set_shot_group", "dg_set_options", "dg_set_mass_mode", "dg_set_op_precision", "dg_num_nodes",
           "dg_node_coords", "dg_face_neighbors", "dg_reference_operator", "dg_device_bytes", "dg_bind",
           "dg_set_fields", "dg_get_fields", "dg_rhs", "dg_step", "dg_energy", "dg_energy_static", "dg_expire_wait", "dg_fma_peak", "dg_stage_times", "dg_autotune", "dg_autotune_layout", "dg_set_launch_variant", "dg_add_receiver", "dg_sample", "dg_save_state",
           "dg_load_state", "dg_adjoint_bytes", "dg_adjoint_bind", "dg_adjoint_reset", "dg_adjoint_inject",
           "dg_adjoint_step", "dg_step_record_bytes", "dg_step_record", "dg_step_record_chain", "dg_adjoint_step_recorded", "dg_adjoint_set", "dg_adjoint_get", "dg_adjoint_gradient", "dg_sync", "dg_time",
           "dg_stable_dt", "dg_last_error", "dg_destroy")

_lib = None


class DGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dgwedge error {code}: {msg}")
        self.code = code


def lib():
    """Load libdgwedge.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not found: the CUDA library has not been built "
                           "(run paper_1607_03399_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "dg_mesh_create": (c_int, [POINTER(P), c_int64, P, c_int64, P, P]),
        "dg_set_order": (c_int, [P, c_int]),
        "dg_set_material": (c_int, [P, P, P]),
        "dg_add_source": (c_int, [P, c_double, c_double, c_double, c_double, c_double, c_double]),
        "dg_set_shots": (c_int, [P, c_int64]),
        "dg_add_shot_source": (c_int, [P, c_int64, c_double, c_double, c_double, c_double, c_double, c_double]),
        "dg_set_shot_order": (c_int, [P, c_int]),
        "dg_set_shot_group": (c_int, [P, c_int64]),
        "dg_set_options": (c_int, [P, c_int, c_int, c_int]),
        "dg_set_mass_mode": (c_int, [P, c_int]),
        "dg_set_op_precision": (c_int, [P, c_int]),
        "dg_num_nodes": (c_int, [P, POINTER(c_int64), POINTER(c_int64)]),
        "dg_node_coords": (c_int, [P, P]),
        "dg_face_neighbors": (c_int, [P, P, POINTER(c_int64)]),
        "dg_reference_operator": (c_int, [P, c_char_p, P, POINTER(c_int64), POINTER(c_int64)]),
        "dg_device_bytes": (c_int, [P, POINTER(c_size_t), POINTER(c_size_t)]),
        "dg_bind": (c_int, [P, P, P, P, P, P]),
        "dg_set_fields": (c_int, [P, P, c_int]),
        "dg_get_fields": (c_int, [P, P, c_int]),
        "dg_rhs": (c_int, [P, P, P]),
        "dg_step": (c_int, [P, c_double, c_int64]),
        "dg_energy": (c_int, [P, POINTER(c_double)]),
        "dg_energy_static": (c_int, [P, P, POINTER(c_double)]),
        "dg_stage_times": (c_int, [P, c_int, POINTER(c_double), POINTER(c_double)]),
        "dg_autotune": (c_int, [P, c_int, POINTER(c_int), POINTER(c_double)]),
        "dg_autotune_layout": (c_int, [P, c_int, POINTER(c_int64), POINTER(c_double)]),
        "dg_set_launch_variant": (c_int, [P, c_int]),
        "dg_add_receiver": (c_int, [P, c_double, c_double, c_double]),
        "dg_sample": (c_int, [P, P]),
        "dg_save_state": (c_int, [P, P]),
        "dg_load_state": (c_int, [P, P, c_double]),
        "dg_adjoint_bytes": (c_int, [P, POINTER(c_size_t)]),
        "dg_adjoint_bind": (c_int, [P, P]),
        "dg_adjoint_reset": (c_int, [P]),
        "dg_adjoint_inject": (c_int, [P, P]),
        "dg_adjoint_step": (c_int, [P, c_double]),
        "dg_step_record_bytes": (c_int, [P, POINTER(c_size_t)]),
        "dg_step_record": (c_int, [P, c_double, P]),
        "dg_step_record_chain": (c_int, [P, c_double, c_int64, P]),
        "dg_adjoint_step_recorded": (c_int, [P, c_double, P]),
        "dg_adjoint_set": (c_int, [P, P, P, c_int]),
        "dg_adjoint_get": (c_int, [P, P, c_int]),
        "dg_adjoint_gradient": (c_int, [P, P, P]),
        "dg_sync": (c_int, [P]),
        "dg_expire_wait": (c_int, [P]),
        "dg_fma_peak": (c_int, [c_int, P, POINTER(c_double)]),
        "dg_time": (c_int, [P, POINTER(c_double)]),
        "dg_stable_dt": (c_int, [P, c_double, POINTER(c_double)]),
        "dg_last_error": (c_char_p, [P]),
        "dg_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(ctx, rc):
    if rc != DG_OK:
        msg = lib().dg_last_error(ctx)
        raise DGError(rc, msg.decode() if msg else "")


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(c_void_p)


# ----------------------------------------------------------------------------
# C-ABI mirrors (host arrays are numpy; device pointers are ints)
# ----------------------------------------------------------------------------

def dg_mesh_create(VX, EToV, etype):
    VX = np.ascontiguousarray(VX, dtype=np.float64)
    EToV = np.ascontiguousarray(EToV, dtype=np.int64)
    etype = np.ascontiguousarray(etype, dtype=np.uint8)
    if EToV.ndim != 2 or EToV.shape[1] != 6 or VX.ndim != 2 or VX.shape[1] != 3 or etype.shape[0] != EToV.shape[0]:
        raise ValueError("VX must be (nv, 3), EToV (K, 6), etype (K,)")
    ctx = c_void_p()
    rc = lib().dg_mesh_create(ctypes.byref(ctx), VX.shape[0], _ptr(VX), EToV.shape[0], _ptr(EToV), _ptr(etype))
    if rc != DG_OK:
        msg = lib().dg_last_error(ctx).decode() if ctx.value else ""
        if ctx.value:
            lib().dg_destroy(ctx)
        raise DGError(rc, msg)
    return ctx


def dg_set_order(ctx, N: int):
    _check(ctx, lib().dg_set_order(ctx, N))


def dg_set_material(ctx, c2, rho):
    c2 = np.ascontiguousarray(c2, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    _check(ctx, lib().dg_set_material(ctx, _ptr(c2), _ptr(rho)))


def dg_add_source(ctx, x: float, y: float, z: float, f0: float, t0: float, amp: float):
    _check(ctx, lib().dg_add_source(ctx, x, y, z, f0, t0, amp))


def dg_set_shots(ctx, shots: int):
    _check(ctx, lib().dg_set_shots(ctx, shots))


def dg_set_shot_order(ctx, order: int):
    _check(ctx, lib().dg_set_shot_order(ctx, order))


def dg_add_shot_source(ctx, shot: int, x, y, z, f0, t0, amp):
    _check(ctx, lib().dg_add_shot_source(ctx, shot, x, y, z, f0, t0, amp))


def dg_set_shot_group(ctx, group: int):
    _check(ctx, lib().dg_set_shot_group(ctx, group))


def dg_set_options(ctx, bc: int, flux: int, precision: int):
    _check(ctx, lib().dg_set_options(ctx, bc, flux, precision))


def dg_set_mass_mode(ctx, mode: int):
    _check(ctx, lib().dg_set_mass_mode(ctx, mode))


def dg_set_op_precision(ctx, mode: int):
    _check(ctx, lib().dg_set_op_precision(ctx, mode))


def dg_num_nodes(ctx):
    w, t = c_int64(), c_int64()
    _check(ctx, lib().dg_num_nodes(ctx, ctypes.byref(w), ctypes.byref(t)))
    return w.value, t.value


def dg_node_coords(ctx):
    w, t = dg_num_nodes(ctx)
    xyz = np.zeros((3, w + t))
    _check(ctx, lib().dg_node_coords(ctx, _ptr(xyz)))
    return xyz


def dg_face_neighbors(ctx):
    n = c_int64()
    _check(ctx, lib().dg_face_neighbors(ctx, None, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.int64)
    _check(ctx, lib().dg_face_neighbors(ctx, _ptr(out), ctypes.byref(n)))
    return out


def dg_reference_operator(ctx, name: str):
    r, c = c_int64(), c_int64()
    _check(ctx, lib().dg_reference_operator(ctx, name.encode(), None, ctypes.byref(r), ctypes.byref(c)))
    out = np.zeros((r.value, c.value))
    _check(ctx, lib().dg_reference_operator(ctx, name.encode(), _ptr(out), ctypes.byref(r), ctypes.byref(c)))
    return out if c.value > 1 else out[:, 0]


def dg_device_bytes(ctx):
    m, f = c_size_t(), c_size_t()
    _check(ctx, lib().dg_device_bytes(ctx, ctypes.byref(m), ctypes.byref(f)))
    return m.value, f.value


def dg_bind(ctx, d_mesh: int, d_q0: int, d_q1: int, d_res: int, stream: int):
    _check(ctx, lib().dg_bind(ctx, c_void_p(d_mesh), c_void_p(d_q0), c_void_p(d_q1), c_void_p(d_res),
                              c_void_p(stream)))


def dg_set_fields(ctx, q, on_device: int):
    _check(ctx, lib().dg_set_fields(ctx, c_void_p(q), on_device))


def dg_get_fields(ctx, q, on_device: int):
    _check(ctx, lib().dg_get_fields(ctx, c_void_p(q), on_device))


def dg_rhs(ctx, d_q: int, d_rhs: int):
    _check(ctx, lib().dg_rhs(ctx, c_void_p(d_q), c_void_p(d_rhs)))


def dg_step(ctx, dt: float, nsteps: int):
    _check(ctx, lib().dg_step(ctx, dt, nsteps))


def dg_energy(ctx) -> float:
    E = c_double()
    _check(ctx, lib().dg_energy(ctx, ctypes.byref(E)))
    return E.value


def dg_energy_static(ctx, d_q: int) -> float:
    E = c_double()
    _check(ctx, lib().dg_energy_static(ctx, c_void_p(d_q), ctypes.byref(E)))
    return E.value


def dg_stage_times(ctx, nrep: int):
    """Mean device microseconds per launch of the wedge and of the tet stage kernel."""
    w, t = c_double(), c_double()
    _check(ctx, lib().dg_stage_times(ctx, nrep, ctypes.byref(w), ctypes.byref(t)))
    return w.value, t.value


def dg_autotune(ctx, nrep: int):
    """(variant, microseconds per wedge-stage launch) of the fastest launch variant, now in use."""
    v, us = c_int(), c_double()
    _check(ctx, lib().dg_autotune(ctx, nrep, ctypes.byref(v), ctypes.byref(us)))
    return v.value, us.value


def dg_set_launch_variant(ctx, variant: int):
    _check(ctx, lib().dg_set_launch_variant(ctx, variant))


def dg_autotune_layout(ctx, nrep: int):
    g, us = c_int64(), c_double()
    _check(ctx, lib().dg_autotune_layout(ctx, nrep, ctypes.byref(g), ctypes.byref(us)))
    return g.value, us.value


def dg_add_receiver(ctx, x, y, z) -> int:
    r = lib().dg_add_receiver(ctx, x, y, z)
    _check(ctx, min(r, 0))
    return r


def dg_sample(ctx, d_out: int):
    _check(ctx, lib().dg_sample(ctx, d_out))


def dg_save_state(ctx, d_dst: int):
    _check(ctx, lib().dg_save_state(ctx, d_dst))


def dg_load_state(ctx, d_src: int, t: float):
    _check(ctx, lib().dg_load_state(ctx, d_src, t))


def dg_adjoint_bytes(ctx) -> int:
    n = c_size_t()
    _check(ctx, lib().dg_adjoint_bytes(ctx, ctypes.byref(n)))
    return n.value


def dg_adjoint_bind(ctx, d_work: int):
    _check(ctx, lib().dg_adjoint_bind(ctx, d_work))


def dg_adjoint_reset(ctx):
    _check(ctx, lib().dg_adjoint_reset(ctx))


def dg_adjoint_inject(ctx, d_resid: int):
    _check(ctx, lib().dg_adjoint_inject(ctx, d_resid))


def dg_adjoint_step(ctx, dt: float):
    _check(ctx, lib().dg_adjoint_step(ctx, dt))


def dg_step_record_bytes(ctx) -> int:
    n = c_size_t()
    _check(ctx, lib().dg_step_record_bytes(ctx, ctypes.byref(n)))
    return n.value


def dg_step_record(ctx, dt: float, d_rec: int):
    _check(ctx, lib().dg_step_record(ctx, dt, d_rec))


def dg_step_record_chain(ctx, dt: float, d_recs):
    """d_recs: sequence of device addresses (int) of the records."""
    arr = (c_void_p * max(1, len(d_recs)))(*[c_void_p(int(x)) for x in d_recs])
    _check(ctx, lib().dg_step_record_chain(ctx, dt, len(d_recs), arr))


def dg_adjoint_step_recorded(ctx, dt: float, d_rec: int):
    _check(ctx, lib().dg_adjoint_step_recorded(ctx, dt, d_rec))


def dg_adjoint_set(ctx, mu_q: int, x: int, on_device: int):
    _check(ctx, lib().dg_adjoint_set(ctx, mu_q, x, on_device))


def dg_adjoint_get(ctx, dst: int, on_device: int):
    _check(ctx, lib().dg_adjoint_get(ctx, dst, on_device))


def dg_adjoint_gradient(ctx, K: int):
    gk, gr = np.zeros(K), np.zeros(K)
    _check(ctx, lib().dg_adjoint_gradient(ctx, gk.ctypes.data, gr.ctypes.data))
    return gk, gr


def dg_expire_wait(ctx):
    _check(ctx, lib().dg_expire_wait(ctx))


def dg_fma_peak(precision: int, stream: int = 0) -> float:
    """Measured CUDA-core FMA throughput of the current device, TFLOP/s."""
    t = c_double()
    rc = lib().dg_fma_peak(precision, c_void_p(stream), ctypes.byref(t))
    if rc != DG_OK:
        raise DGError(rc, "dg_fma_peak failed")
    return t.value


def dg_sync(ctx):
    _check(ctx, lib().dg_sync(ctx))


def dg_time(ctx) -> float:
    t = c_double()
    _check(ctx, lib().dg_time(ctx, ctypes.byref(t)))
    return t.value


def dg_stable_dt(ctx, cfl: float) -> float:
    dt = c_double()
    _check(ctx, lib().dg_stable_dt(ctx, cfl, ctypes.byref(dt)))
    return dt.value


def dg_destroy(ctx):
    if ctx is not None and ctx.value:
        lib().dg_destroy(ctx)


# ----------------------------------------------------------------------------
# convenience wrapper with torch-owned device memory
# ----------------------------------------------------------------------------

BC = {"dirichlet": DG_BC_DIRICHLET, "rigid": DG_BC_RIGID}
FLUX = {"upwind": DG_FLUX_UPWIND, "central": DG_FLUX_CENTRAL}
PREC = {"f32": DG_F32, "f64": DG_F64}
MASS = {"onthefly": DG_MASS_ONTHEFLY, "stored": DG_MASS_STORED}
OPS = {"fp32": DG_OPS_FP32, "tf32x3": DG_OPS_TF32X3, "tf32": DG_OPS_TF32, "bf16": DG_OPS_BF16}


class Solver:
    """One mesh, one order, bound to one CUDA device and stream.

    Device memory (mesh blob, two state buffers, residual) is allocated as
    torch uint8 tensors and handed to the library by pointer.  With shots > 1
    the state arrays are [shots][4][total_nodes] (else [4][total_nodes]);
    `sources` go into every shot, `shot_sources` ((shot, x, y, z, f0, t0, amp))
    into one."""

    def __init__(self, VX, EToV, etype, N: int, c2=None, rho=None, bc: str = "rigid", flux: str = "upwind",
                 precision: str = "f32", device: str = "cuda:0", stream=None, sources=(), mass: str = "stored",
                 shots: int = 1, shot_sources=(), receivers=(), shot_order: str = "outer", ops: str = "fp32"):
        import torch
        self.torch = torch
        self.ctx = dg_mesh_create(VX, EToV, etype)
        try:
            dg_set_order(self.ctx, N)
            K = np.asarray(EToV).shape[0]
            if c2 is not None or rho is not None:
                dg_set_material(self.ctx, np.ones(K) if c2 is None else c2, np.ones(K) if rho is None else rho)
            dg_set_options(self.ctx, BC[bc], FLUX[flux], PREC[precision])
            dg_set_mass_mode(self.ctx, MASS[mass])
            dg_set_op_precision(self.ctx, OPS[ops])
            dg_set_shots(self.ctx, shots)
            if isinstance(shot_order, str):
                dg_set_shot_order(self.ctx, {"outer": DG_SHOTS_OUTER, "inner": DG_SHOTS_INNER}[shot_order])
            else:  # shots per group
                dg_set_shot_group(self.ctx, int(shot_order))
            self.shots = shots
            for src in sources:       # (x, y, z, f0, t0, amp)
                dg_add_source(self.ctx, *src)
            for src in shot_sources:  # (shot, x, y, z, f0, t0, amp)
                dg_add_shot_source(self.ctx, *src)
            self.nrec = 0
            for rc in receivers:      # (x, y, z)
                dg_add_receiver(self.ctx, *rc)
                self.nrec += 1
            self.K = K
            self.N = N
            self.precision = precision
            self.dtype = torch.float32 if precision == "f32" else torch.float64
            self.np_dtype = np.float32 if precision == "f32" else np.float64
            self.wedge_nodes, self.tet_nodes = dg_num_nodes(self.ctx)
            self.total_nodes = self.wedge_nodes + self.tet_nodes
            self.field_shape = (4, self.total_nodes) if shots == 1 else (shots, 4, self.total_nodes)
            self.device = torch.device(device)
            mb, fb = dg_device_bytes(self.ctx)
            self.mesh_bytes, self.field_bytes = mb, fb
            with torch.cuda.device(self.device):
                self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
                self.d_mesh = torch.empty(mb, dtype=torch.uint8, device=self.device)
                self.d_q0 = torch.empty(fb, dtype=torch.uint8, device=self.device)
                self.d_q1 = torch.empty(fb, dtype=torch.uint8, device=self.device)
                self.d_res = torch.empty(fb, dtype=torch.uint8, device=self.device)
                torch.cuda.current_stream(self.device).synchronize()
                dg_bind(self.ctx, self.d_mesh.data_ptr(), self.d_q0.data_ptr(), self.d_q1.data_ptr(),
                        self.d_res.data_ptr(), self.stream.cuda_stream)
        except Exception:
            dg_destroy(self.ctx)
            self.ctx = None
            raise

    # -- state ------------------------------------------------------------
    def node_coords(self):
        return dg_node_coords(self.ctx)

    def set_fields(self, q):
        """q: numpy [4][total_nodes] (host) or a torch tensor on the device."""
        t = self.torch
        if isinstance(q, t.Tensor) and q.is_cuda:
            q = q.to(self.dtype).contiguous()
            self._wait_torch()
            dg_set_fields(self.ctx, q.data_ptr(), 1)
            self._keep = q
        else:
            qh = np.ascontiguousarray(q, dtype=self.np_dtype)
            assert qh.shape == self.field_shape
            dg_set_fields(self.ctx, qh.ctypes.data, 0)

    def get_fields(self, device: bool = False):
        if device:
            out = self.torch.empty(self.field_shape, dtype=self.dtype, device=self.device)
            dg_get_fields(self.ctx, out.data_ptr(), 1)
            self.stream.synchronize()
            return out
        out = np.empty(self.field_shape, dtype=self.np_dtype)
        dg_get_fields(self.ctx, out.ctypes.data, 0)
        return out

    def rhs(self, q):
        """Semi-discrete right-hand side of a state q (numpy or device tensor)."""
        t = self.torch
        if isinstance(q, t.Tensor) and q.is_cuda:
            dq = q.to(self.dtype).contiguous()
        else:
            dq = t.from_numpy(np.ascontiguousarray(q, dtype=self.np_dtype)).to(self.device)
        out = t.empty_like(dq)
        self._wait_torch()
        dg_rhs(self.ctx, dq.data_ptr(), out.data_ptr())
        self.stream.synchronize()
        return out

    def step(self, dt: float, nsteps: int):
        dg_step(self.ctx, dt, nsteps)

    def stage_times(self, nrep: int = 20):
        """(wedge, tet) mean microseconds per stage-kernel launch; the state is unchanged."""
        self._wait_torch()
        return dg_stage_times(self.ctx, nrep)

    def autotune(self, nrep: int = 10):
        """Pick the fastest wedge-stage launch variant: returns (blocks per CTA,
        factor in stage?, split over field pairs?, us)."""
        self._wait_torch()
        v, us = dg_autotune(self.ctx, nrep)
        return (v >> 1) & 3, bool(v & 1), bool(v & 8), us

    # -- receivers, checkpoints, adjoint ------------------------------------
    def autotune_layout(self, nrep: int = 10):
        """Pick the shots-per-group layout by timing (resets the state to zero):
        returns (shots per group, us per stage)."""
        self._wait_torch()
        return dg_autotune_layout(self.ctx, nrep)

    def sample(self, out):
        """Pressure at the receivers into the device tensor out[shots][receivers]."""
        self._wait_torch()
        dg_sample(self.ctx, out.data_ptr())

    def save_state(self, buf=None):
        """Device copy of the packed current state (a checkpoint)."""
        if buf is None:
            buf = self.torch.empty(self.field_bytes, dtype=self.torch.uint8, device=self.device)
        dg_save_state(self.ctx, buf.data_ptr())
        return buf

    def load_state(self, buf, t: float):
        dg_load_state(self.ctx, buf.data_ptr(), t)

    def adjoint_bind(self):
        n = dg_adjoint_bytes(self.ctx)
        self.d_adj = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
        self.stream.synchronize()
        dg_adjoint_bind(self.ctx, self.d_adj.data_ptr())

    def adjoint_reset(self):
        dg_adjoint_reset(self.ctx)

    def adjoint_inject(self, resid):
        dg_adjoint_inject(self.ctx, resid.data_ptr())

    def adjoint_step(self, dt: float):
        dg_adjoint_step(self.ctx, dt)

    def new_record(self):
        """Device buffer for one step record (dg_step_record)."""
        return self.torch.empty(dg_step_record_bytes(self.ctx), dtype=self.torch.uint8, device=self.device)

    def step_record(self, dt: float, rec):
        """One step that also writes its stage inputs and right-hand sides to rec."""
        self._wait_torch()
        dg_step_record(self.ctx, dt, rec.data_ptr())

    def step_record_chain(self, dt: float, recs):
        """len(recs) steps, step i's stage inputs and right-hand sides into recs[i]
        (dg_step_record_chain)."""
        self._wait_torch()
        dg_step_record_chain(self.ctx, dt, [r.data_ptr() for r in recs])

    def adjoint_step_recorded(self, dt: float, rec):
        dg_adjoint_step_recorded(self.ctx, dt, rec.data_ptr())

    def adjoint_set(self, mu_q, x):
        """mu_q, x: numpy arrays of the field shape."""
        a = np.ascontiguousarray(mu_q, dtype=self.np_dtype)
        b = np.ascontiguousarray(x, dtype=self.np_dtype)
        dg_adjoint_set(self.ctx, a.ctypes.data, b.ctypes.data, 0)

    def adjoint_get(self):
        out = np.empty(self.field_shape, dtype=self.np_dtype)
        dg_adjoint_get(self.ctx, out.ctypes.data, 0)
        return out

    def adjoint_gradient(self):
        """(dJ/dkappa, dJ/drho) per element, input order."""
        return dg_adjoint_gradient(self.ctx, self.K)

    def energy(self) -> float:
        return dg_energy(self.ctx)

    def sync(self):
        dg_sync(self.ctx)

    def time(self) -> float:
        return dg_time(self.ctx)

    def stable_dt(self, cfl: float) -> float:
        return dg_stable_dt(self.ctx, cfl)

    def _wait_torch(self):
        # order the library's stream after work queued on torch's current stream
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))

    def close(self):
        if getattr(self, "ctx", None) is not None:
            try:
                self.stream.synchronize()
            finally:
                dg_destroy(self.ctx)
                self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostMesh:
    """Host-only view of a mesh context (no GPU needed): connectivity, node
    coordinates, reference operators, stable time step."""

    def __init__(self, VX, EToV, etype, N: int, c2=None, rho=None):
        self.ctx = dg_mesh_create(VX, EToV, etype)
        try:
            dg_set_order(self.ctx, N)
            if c2 is not None:
                dg_set_material(self.ctx, c2, rho)
        except Exception:
            dg_destroy(self.ctx)
            raise
        self.wedge_nodes, self.tet_nodes = dg_num_nodes(self.ctx)

    def node_coords(self):
        return dg_node_coords(self.ctx)

    def face_neighbors(self):
        return dg_face_neighbors(self.ctx)

    def operator(self, name):
        return dg_reference_operator(self.ctx, name)

    def stable_dt(self, cfl):
        return dg_stable_dt(self.ctx, cfl)

    def __del__(self):
        try:
            dg_destroy(self.ctx)
        except Exception:
            pass
