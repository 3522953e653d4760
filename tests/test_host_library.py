"""CPU tests of the C-ABI library's host side (no GPU calls): the shared
library loads and exports every entry point declared in include/dgwedge.h,
its independently built reference operators, node coordinates, face-node
connectivity and stable time step agree with the oracle, and invalid meshes
or call orders are rejected with the documented status codes."""
import os
import re

import numpy as np
import pytest

from oracle import reference as R
from oracle.dg import Solver as OracleSolver
from paper_1607_03399_gb300 import dg
from paper_1607_03399_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "dgwedge.h")).read()
    declared = set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", hdr))
    L = dg.lib()
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(dg.EXPORTS)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5])
def test_reference_operators_match_oracle(N):
    m = I.cube_wavy_mesh(1, 1, 0.0)
    H = dg.HostMesh(m.VX, m.EToV, m.etype, N)
    tri, line, tet = R.Triangle(N), R.Line(N), R.Tet(N)
    assert np.allclose(H.operator("tri.r"), tri.x[:, 0], atol=1e-14)
    assert np.allclose(H.operator("tri.s"), tri.x[:, 1], atol=1e-14)
    assert np.allclose(H.operator("line.r"), line.x, atol=1e-15)
    for name, ref in (("tri.Dr", tri.Dr), ("tri.Ds", tri.Ds), ("tri.M", tri.M), ("tri.M0", tri.Ma[0]),
                      ("tri.M1", tri.Ma[1]), ("tri.M2", tri.Ma[2]), ("line.D", line.D), ("line.M", line.M),
                      ("line.Ma", line.Ma), ("line.Mb", line.Mb), ("tet.Dr", tet.Dr), ("tet.Ds", tet.Ds),
                      ("tet.Dt", tet.Dt), ("tet.M", tet.M)):
        got = H.operator(name)
        assert np.allclose(got, ref, atol=1e-12 * max(1.0, np.abs(ref).max())), name
    assert np.allclose(H.operator("line.ell0"), line.ell0, atol=1e-12)
    assert np.allclose(H.operator("line.ellN"), line.ellN, atol=1e-12)
    assert np.allclose(H.operator("tet.r"), tet.x[:, 0], atol=1e-14)
    assert np.allclose(H.operator("tet.s"), tet.x[:, 1], atol=1e-14)
    assert np.allclose(H.operator("tet.t"), tet.x[:, 2], atol=1e-14)
    # reference lift of every tet face: M^-1 E_f M^tri
    Minv = np.linalg.inv(tet.M)
    lift = np.concatenate([Minv[:, tet.faces[f]] @ tri.M for f in range(4)], axis=1)
    # two independent inversions of the tet mass (condition number 250 at N = 4,
    # 360 at N = 5): agreement relative to the largest entry
    assert np.allclose(H.operator("tet.LIFT"), lift, atol=4e-12 * np.abs(lift).max())


MESHES = {
    "wavy": lambda: I.cube_wavy_mesh(3, 3, 0.05),
    "bumpy": lambda: I.bumpy_layered_mesh(3, 4),
    "hybrid": lambda: I.hybrid_mesh(3, 2, 2),
    "tets": lambda: I.tet_box_mesh(2, 2),
}


@pytest.mark.parametrize("meshname", list(MESHES))
@pytest.mark.parametrize("N", [1, 3, 4])
def test_nodes_and_face_neighbours_match_oracle(meshname, N):
    m = MESHES[meshname]()
    H = dg.HostMesh(m.VX, m.EToV, m.etype, N)
    S = OracleSolver(m.VX, m.EToV, m.etype, N)
    C = S.conn
    assert H.wedge_nodes + H.tet_nodes == C.total_nodes
    assert np.allclose(H.node_coords(), C.xyz, atol=1e-13)
    nb = H.face_neighbors()
    expect = []
    for k in range(C.K):
        for f in range(C.nfaces(k)):
            gP = C.vmapP[(k, f)].copy()
            if C.EToE[k, f] < 0:
                gP[:] = -1
            expect.append(gP)
    assert np.array_equal(nb, np.concatenate(expect))


@pytest.mark.parametrize("meshname", ["wavy", "hybrid"])
def test_stable_dt_matches_oracle(meshname):
    m = MESHES[meshname]()
    c2, rho = I.random_material(m.K, 2, 1.0, 3.0, 1.0, 2.0)
    H = dg.HostMesh(m.VX, m.EToV, m.etype, 3, c2, rho)
    S = OracleSolver(m.VX, m.EToV, m.etype, 3, c2, rho)
    assert abs(H.stable_dt(0.5) - S.stable_dt(0.5)) < 1e-14 * S.stable_dt(0.5)


def _expect_error(code, fn):
    with pytest.raises(dg.DGError) as ei:
        fn()
    assert ei.value.code == code, str(ei.value)
    return str(ei.value)


def test_invalid_meshes_are_rejected():
    m = I.cube_wavy_mesh(2, 2, 0.0)
    # top vertex moved sideways: not vertically mapped
    VX = m.VX.copy()
    VX[m.EToV[3, 3], 0] += 0.01
    msg = _expect_error(dg.DG_ERR_MESH, lambda: dg.dg_mesh_create(VX, m.EToV, m.etype))
    assert "vertically mapped" in msg
    # clockwise bottom triangle: J < 0
    E = m.EToV.copy()
    E[5, [1, 2]] = E[5, [2, 1]]
    E[5, [4, 5]] = E[5, [5, 4]]
    _expect_error(dg.DG_ERR_MESH, lambda: dg.dg_mesh_create(m.VX, E, m.etype))
    # vertex id out of range
    E = m.EToV.copy()
    E[0, 0] = m.VX.shape[0]
    _expect_error(dg.DG_ERR_MESH, lambda: dg.dg_mesh_create(m.VX, E, m.etype))
    # a face shared by three elements
    E = np.vstack([m.EToV, m.EToV[:1]])
    t = np.concatenate([m.etype, m.etype[:1]])
    _expect_error(dg.DG_ERR_MESH, lambda: dg.dg_mesh_create(m.VX, E, t))
    # negative tet
    tm = I.tet_box_mesh(1, 1)
    E = tm.EToV.copy()
    E[0, [1, 2]] = E[0, [2, 1]]
    _expect_error(dg.DG_ERR_MESH, lambda: dg.dg_mesh_create(tm.VX, E, tm.etype))
    # unknown element type
    t = m.etype.copy()
    t[0] = 5
    _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_mesh_create(m.VX, m.EToV, t))


def test_call_order_and_argument_errors():
    m = I.cube_wavy_mesh(2, 2, 0.0)
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_num_nodes(ctx))
        _expect_error(dg.DG_ERR_ORDER, lambda: dg.dg_set_order(ctx, 0))
        _expect_error(dg.DG_ERR_ORDER, lambda: dg.dg_set_order(ctx, 6))
        dg.dg_set_order(ctx, 2)
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_set_options(ctx, 7, 0, 0))
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_set_material(ctx, -np.ones(m.K), np.ones(m.K)))
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_step(ctx, 0.1, 1))
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_autotune(ctx, 2))
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_stage_times(ctx, 2))
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_energy(ctx))
        buf = np.zeros(8)
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_set_fields(ctx, buf.ctypes.data, 0))
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_bind(ctx, 0, 0, 0, 0, 0))
        mb, fb = dg.dg_device_bytes(ctx)
        assert mb > 0 and fb >= 4 * 4 * dg.dg_num_nodes(ctx)[0]
        dg.dg_set_options(ctx, dg.DG_BC_DIRICHLET, dg.DG_FLUX_CENTRAL, dg.DG_F64)
        mb2, fb2 = dg.dg_device_bytes(ctx)
        assert fb2 == 2 * fb
        # stored mass factors: Nt (Nt + 1) / 2 reals per (padded) wedge in the mesh blob
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_set_mass_mode(ctx, 2))
        dg.dg_set_mass_mode(ctx, dg.DG_MASS_ONTHEFLY)
        mb3, fb3 = dg.dg_device_bytes(ctx)
        dg.dg_set_mass_mode(ctx, dg.DG_MASS_STORED)
        mb4, fb4 = dg.dg_device_bytes(ctx)
        assert fb3 == fb4 == fb2 and mb4 == mb2
        nl4 = (6 * 7 // 2 + 3) // 4  # the packed factor in groups of four entries per lane
        assert mb4 - mb3 >= 32 * 4 * nl4 * 8 and mb4 - mb3 < 32 * 4 * nl4 * 8 + 256
    finally:
        dg.dg_destroy(ctx)


def test_shots_arguments_and_sizes():
    """dg_set_shots: validation, call order, and the state buffers holding every shot."""
    m = I.cube_wavy_mesh(2, 2, 0.0)
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_set_shots(ctx, 2))
        dg.dg_set_order(ctx, 2)
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_set_shots(ctx, 0))
        mb1, fb1 = dg.dg_device_bytes(ctx)
        dg.dg_set_shots(ctx, 5)
        mb5, fb5 = dg.dg_device_bytes(ctx)
        wn, _ = dg.dg_num_nodes(ctx)
        assert fb5 >= 5 * 4 * 4 * wn and fb5 > fb1 and mb5 > mb1
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_add_shot_source(ctx, 5, 0.5, 0.5, 0.5, 5.0, 0.1, 1.0))
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_add_shot_source(ctx, -1, 0.5, 0.5, 0.5, 5.0, 0.1, 1.0))
        dg.dg_add_shot_source(ctx, 4, 0.5, 0.5, 0.5, 5.0, 0.1, 1.0)
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_set_shots(ctx, 4))   # would orphan the shot-4 source
        dg.dg_set_shots(ctx, 6)
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_set_shot_order(ctx, 2))
        dg.dg_set_shot_order(ctx, dg.DG_SHOTS_INNER)
        _, fb6 = dg.dg_device_bytes(ctx)
        dg.dg_set_shot_order(ctx, dg.DG_SHOTS_OUTER)
        assert dg.dg_device_bytes(ctx)[1] == fb6   # the order changes no buffer size
    finally:
        dg.dg_destroy(ctx)


def test_step_record_arguments_and_size():
    """Stage records: ten packed fields; null or misaligned records, dt <= 0 and
    unbound contexts or adjoints are refused before any device work."""
    m = I.cube_wavy_mesh(2, 2, 0.0)
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_step_record_bytes(ctx))
        dg.dg_set_order(ctx, 3)
        dg.dg_set_shots(ctx, 3)
        _, fb = dg.dg_device_bytes(ctx)
        assert dg.dg_step_record_bytes(ctx) == 10 * fb
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_step_record(ctx, 0.1, 0))
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_step_record(ctx, 0.1, 4096 + 16))
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_step_record(ctx, 0.0, 4096))
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_step_record(ctx, 0.1, 4096))
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_step_record_chain(ctx, 0.1, [4096, 0]))
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_step_record_chain(ctx, 0.1, [4096, 4096 + 64]))
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_step_record_chain(ctx, 0.1, [4096, 8192]))
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_step_record_chain(ctx, 0.1, []))
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_adjoint_step_recorded(ctx, 0.1, 0))
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_adjoint_step_recorded(ctx, -1.0, 4096))
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_adjoint_step_recorded(ctx, 0.1, 4096))
    finally:
        dg.dg_destroy(ctx)


def test_empty_mesh_and_table_limits():
    """Degenerate and maximum sizes on the host side: a mesh with no elements is
    refused; the (source, shot) table stops at 4096 entries and the receiver
    table at 65536, each with DG_ERR_ARG and the context still usable."""
    m = I.cube_wavy_mesh(2, 1, 0.0)
    _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_mesh_create(m.VX, m.EToV[:0], m.etype[:0]))
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        dg.dg_set_order(ctx, 1)
        dg.dg_set_shots(ctx, 2)
        for _ in range(2048):  # each source goes into both shots
            dg.dg_add_source(ctx, 0.5, 0.5, 0.5, 5.0, 0.0, 1.0)
        msg = _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_add_shot_source(ctx, 1, 0.5, 0.5, 0.5, 5.0, 0.0, 1.0))
        assert "too many sources" in msg
        for i in range(65536):
            assert dg.dg_add_receiver(ctx, 0.25 + (i % 7) * 0.05, 0.5, 0.5) == i
        msg = _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_add_receiver(ctx, 0.5, 0.5, 0.5))
        assert "too many receivers" in msg
        _, fb = dg.dg_device_bytes(ctx)
        assert fb > 0
    finally:
        dg.dg_destroy(ctx)


def test_adjoint_workspace_size():
    """dg_adjoint_bytes: fourteen packed fields plus the FP64 gradient sums of every
    device element (wedges and tets, padded blocks) and five face sums per
    wedge, computable before dg_bind."""
    m = I.hybrid_mesh(3, 2, 1)
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        _expect_error(dg.DG_ERR_STATE, lambda: dg.dg_adjoint_bytes(ctx))
        dg.dg_set_order(ctx, 2)
        dg.dg_set_shots(ctx, 3)
        _, fb = dg.dg_device_bytes(ctx)
        nw, nt = int((m.etype == 6).sum()) * 3, int((m.etype == 4).sum()) * 3
        def pad(n):
            return (n + 31) // 32 * 32 * 8 + 255 & ~255
        assert dg.dg_adjoint_bytes(ctx) == 14 * fb + 7 * pad(nw) + 2 * pad(nt)
    finally:
        dg.dg_destroy(ctx)


def test_merge_meshes_keeps_pieces_apart():
    a, b = I.cube_wavy_mesh(2, 2, 0.02), I.hybrid_mesh(2, 1, 1)
    m = I.merge_meshes([a, b])
    assert m.K == a.K + b.K and m.meta["offsets"] == [0, a.K]
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        dg.dg_set_order(ctx, 1)
        wn, tn = dg.dg_num_nodes(ctx)
        nb = dg.dg_face_neighbors(ctx)
        # N = 1: a wedge has 2 x 3 + 3 x 4 face nodes, a tet 4 x 3; nodes of piece a come first
        per = np.where(m.etype == I.WEDGE, 18, 12)
        Ta = 6 * a.K
        split = int(per[: a.K].sum())
        assert nb.size == per.sum() and (nb[:split] < Ta).all() and (nb[split:][nb[split:] >= 0] >= Ta).all()
    finally:
        dg.dg_destroy(ctx)


def _in_block_fractions(m):
    """Fraction of interior triangle-face and quad-face neighbours that lie in the
    same 32-element block (their traces come from the block's shared-memory slab)."""
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        dg.dg_set_order(ctx, 1)
        nb = dg.dg_face_neighbors(ctx).reshape(m.K, 18)
    finally:
        dg.dg_destroy(ctx)
    k = np.arange(m.K)[:, None]
    tri = nb[:, [0, 3]] // 6
    quad = nb[:, [6, 10, 14]] // 6
    ft = (tri[nb[:, [0, 3]] >= 0] // 32 == np.broadcast_to(k, tri.shape)[nb[:, [0, 3]] >= 0] // 32).mean()
    fq = (quad[nb[:, [6, 10, 14]] >= 0] // 32 == np.broadcast_to(k, quad.shape)[nb[:, [6, 10, 14]] >= 0] // 32).mean()
    return ft, fq


def test_column_order_keeps_vertical_traces_in_the_block():
    """Column-major order with 16 layers: a 32-element block holds two whole
    columns, so every vertical (triangle-face) neighbour is in the same block --
    the layer-marching reuse of vertical traces, through shared memory."""
    ft, fq = _in_block_fractions(I.bumpy_layered_mesh(8, 16))
    assert ft == 1.0
    assert 0.2 < fq < 0.5
    # the comparison order: the same mesh layer by layer keeps none of them
    lm, perm = I.layer_major(I.bumpy_layered_mesh(8, 16), 16)
    assert sorted(perm.tolist()) == list(range(lm.K))
    ft, fq = _in_block_fractions(lm)
    assert ft == 0.0


def test_op_precision_needs_fp32_fields():
    m = I.cube_wavy_mesh(2, 2, 0.0)
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        dg.dg_set_order(ctx, 3)
        dg.dg_set_options(ctx, dg.DG_BC_RIGID, dg.DG_FLUX_UPWIND, dg.DG_F64)
        with pytest.raises(dg.DGError) as ei:
            dg.dg_set_op_precision(ctx, dg.DG_OPS_TF32)
        assert ei.value.code == dg.DG_ERR_ARG
        dg.dg_set_op_precision(ctx, dg.DG_OPS_FP32)
    finally:
        dg.dg_destroy(ctx)


def test_shot_group_must_divide_the_shots():
    m = I.cube_wavy_mesh(2, 2, 0.0)
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        dg.dg_set_order(ctx, 2)
        dg.dg_set_shots(ctx, 6)
        for bad in (0, 4, 5):
            with pytest.raises(dg.DGError) as ei:
                dg.dg_set_shot_group(ctx, bad)
            assert ei.value.code == dg.DG_ERR_ARG
        for good in (1, 2, 3, 6):
            dg.dg_set_shot_group(ctx, good)
        with pytest.raises(dg.DGError) as ei:
            dg.dg_set_shots(ctx, 4)  # 6 shots per group no longer divides
        assert ei.value.code == dg.DG_ERR_ARG
    finally:
        dg.dg_destroy(ctx)


def test_order_5_limits():
    """N = 5 is accepted; the tensor-core applies (a slice must fit one
    16-row tile, Nt = 21 here) are refused at bind time only, so this host
    check stops at the order."""
    m = I.cube_wavy_mesh(1, 1, 0.0)
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        dg.dg_set_order(ctx, 5)
        assert dg.dg_num_nodes(ctx)[0] == m.K * 6 * 21
    finally:
        dg.dg_destroy(ctx)


def test_launch_variant_encoding():
    """dg_set_launch_variant takes the encoding dg_autotune reports: bit 0 the
    factor recomputed, bits 1-2 blocks per CTA (1, or 2 for FP32 at N = 3),
    bit 3 the field-pair split stage (stored factor, one block per CTA)."""
    m = I.cube_wavy_mesh(2, 1, 0.0)
    ctx = dg.dg_mesh_create(m.VX, m.EToV, m.etype)
    try:
        dg.dg_set_order(ctx, 3)
        for v in (2, 3, 4, 5, 10):
            dg.dg_set_launch_variant(ctx, v)
        for v in (0, 1, 6, 7, 11, 12, 16, 18):
            _expect_error(dg.DG_ERR_ARG, lambda v=v: dg.dg_set_launch_variant(ctx, v))
        dg.dg_set_order(ctx, 4)
        _expect_error(dg.DG_ERR_ARG, lambda: dg.dg_set_launch_variant(ctx, 4))
    finally:
        dg.dg_destroy(ctx)
