"""Seeded synthetic inputs: layered wedge meshes, hybrid wedge/tet meshes,
per-element materials and random field states.

This module produces vertex coordinates, element-to-vertex lists, element
types and plain arrays only.  It contains none of the discretisation's
arithmetic (no basis, no geometric factors, no fluxes), so both the CUDA path
and the CPU oracle can take their inputs from it.

Layered meshes follow Section 5 of the paper: a surface triangulation of a
rectangle is extruded through layers whose interfaces are surfaces
z_k(x, y); every wedge is vertically mapped (its three vertex pairs share
x and y).  Element order is column-major (all layers of one triangle column
are consecutive), which is the order the GPU kernels are tuned for.

Vertex convention for a wedge: EToV[k] = (b0, b1, b2, t0, t1, t2), bottom
triangle counter-clockwise seen from +z, t_a directly above b_a.
Tetrahedra use the first four entries and -1 for the rest.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

WEDGE = 6
TET = 4


@dataclass
class Mesh:
    """Plain mesh arrays (the C-ABI's dg_mesh_create arguments)."""

    VX: np.ndarray            # (nverts, 3) float64
    EToV: np.ndarray          # (K, 6) int64, tets padded with -1
    etype: np.ndarray         # (K,) uint8, WEDGE or TET
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def K(self) -> int:
        return int(self.EToV.shape[0])


def _grid_triangles(nx: int, ny: int):
    """Split each cell of an nx x ny grid of squares along the (i,j)->(i+1,j+1)
    diagonal into two counter-clockwise triangles.  Returns (ntri, 3) indices
    into the (nx+1) x (ny+1) grid points (point id = j*(nx+1) + i)."""
    tris = []
    for j in range(ny):
        for i in range(nx):
            p00 = j * (nx + 1) + i
            p10 = p00 + 1
            p01 = p00 + (nx + 1)
            p11 = p01 + 1
            tris.append((p00, p10, p11))
            tris.append((p00, p11, p01))
    return np.asarray(tris, dtype=np.int64)


def layered_wedge_mesh(nx: int, ny: int, nlayers: int, interface,
                       box=(0.0, 1.0, 0.0, 1.0), name: str = "") -> Mesh:
    """Extrude the nx x ny two-triangles-per-square footprint through
    `nlayers` layers.  `interface(k, x, y)` returns z of layer interface k
    (k = 0 .. nlayers) at the footprint points (arrays)."""
    x0, x1, y0, y1 = box
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    X, Y = np.meshgrid(xs, ys)               # (ny+1, nx+1)
    px = X.ravel()
    py = Y.ravel()
    npts = px.size
    L1 = nlayers + 1
    # column-major vertices: vertex id = point * (nlayers+1) + k
    VX = np.zeros((npts * L1, 3))
    for k in range(L1):
        z = np.asarray(interface(k, px, py), dtype=np.float64)
        VX[k::L1, 0] = px
        VX[k::L1, 1] = py
        VX[k::L1, 2] = z
    tris = _grid_triangles(nx, ny)
    ntri = tris.shape[0]
    EToV = np.zeros((ntri * nlayers, 6), dtype=np.int64)
    for l in range(nlayers):
        EToV[l::nlayers, 0:3] = tris * L1 + l
        EToV[l::nlayers, 3:6] = tris * L1 + l + 1
    etype = np.full(ntri * nlayers, WEDGE, dtype=np.uint8)
    return Mesh(VX, EToV, etype, name=name,
                meta=dict(nx=nx, ny=ny, nlayers=nlayers, ntri=ntri))


def cube_wavy_mesh(m: int = 4, nlayers: int = 4, amp: float = 0.03) -> Mesh:
    """[0,1]^3, m x m squares split into 2m^2 right triangles, `nlayers`
    layers.  Interior interfaces z_k = k/L + amp sin(2 pi x) sin(2 pi y),
    flat top and bottom.  m=4, L=4 gives the 128-wedge FP64 test case."""
    def iface(k, x, y):
        z = np.full_like(x, k / nlayers)
        if 0 < k < nlayers:
            z = z + amp * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
        return z
    return layered_wedge_mesh(m, m, nlayers, iface,
                              name=f"cube_wavy_{m}x{m}x{nlayers}")


def _bump_field(seed: int, nbumps: int = 8):
    """Sum of `nbumps` Gaussian bumps on [0,1]^2 with seeded centres, widths
    and signs, normalised to max |B| = 1 on a fine grid."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, size=(nbumps, 2))
    w = rng.uniform(0.1, 0.3, size=nbumps)
    sg = rng.choice([-1.0, 1.0], size=nbumps)

    def raw(x, y):
        out = np.zeros_like(np.asarray(x, dtype=np.float64))
        for b in range(nbumps):
            r2 = (x - c[b, 0]) ** 2 + (y - c[b, 1]) ** 2
            out = out + sg[b] * np.exp(-r2 / (w[b] ** 2))
        return out

    g = np.linspace(0.0, 1.0, 257)
    GX, GY = np.meshgrid(g, g)
    scale = float(np.max(np.abs(raw(GX, GY))))
    return lambda x, y: raw(x, y) / scale


def bumpy_layered_mesh(ntri_side: int, nlayers: int, amp_frac: float = 0.2,
                       seed0: int = 1000, name: str = "") -> Mesh:
    """[0,1]^3 footprint of 2*ntri_side^2 triangles, `nlayers` layers, each
    interior interface z_k = k/L + amp_frac*(1/L)*B_k(x,y) where B_k is a
    seeded sum of Gaussian bumps (seed seed0+k); flat top and bottom.
    ntri_side=128, nlayers=16 gives the 524288-wedge throughput workload."""
    bumps = {k: _bump_field(seed0 + k) for k in range(1, nlayers)}

    def iface(k, x, y):
        z = np.full_like(x, k / nlayers, dtype=np.float64)
        if 0 < k < nlayers:
            z = z + amp_frac / nlayers * bumps[k](x, y)
        return z
    return layered_wedge_mesh(ntri_side, ntri_side, nlayers, iface,
                              name=name or f"bumpy_{ntri_side}x{ntri_side}x{nlayers}")


def perturbed_layered_mesh(m: int, nlayers: int, frac: float, seed: int,
                           box=(-1.0, 1.0, -1.0, 1.0), zrange=(-1.0, 1.0)) -> Mesh:
    """Layered mesh whose interior interface vertices are moved vertically by
    U(-frac, frac) * layer height (seeded); top and bottom stay flat.  On the
    bi-unit cube this is the 'randomly perturbed vertically mapped wedges'
    family used for unstructured refinement and the spectrum experiment."""
    rng = np.random.default_rng(seed)
    z0, z1 = zrange
    hL = (z1 - z0) / nlayers
    npts = (m + 1) * (m + 1)
    pert = rng.uniform(-frac, frac, size=(nlayers + 1, npts)) * hL

    def iface(k, x, y):
        z = np.full_like(x, z0 + k * hL, dtype=np.float64)
        if 0 < k < nlayers:
            z = z + pert[k]
        return z
    return layered_wedge_mesh(m, m, nlayers, iface, box=box,
                              name=f"perturbed_{m}x{m}x{nlayers}_s{seed}")


def _prism_to_tets(v):
    """Split one prism (bottom v0 v1 v2, top v3 v4 v5, v_{a+3} above v_a)
    into three tetrahedra such that every quadrilateral face is cut by the
    diagonal through its lowest global vertex id; neighbouring prisms then
    cut their shared quad face the same way, so the tet mesh is conforming."""
    v = list(v)
    # rotate / mirror the prism so that its minimum-id vertex is local 0
    imin = int(np.argmin(v))
    rot = {0: (0, 1, 2, 3, 4, 5), 1: (1, 2, 0, 4, 5, 3), 2: (2, 0, 1, 5, 3, 4),
           3: (3, 5, 4, 0, 2, 1), 4: (4, 3, 5, 1, 0, 2), 5: (5, 4, 3, 2, 1, 0)}[imin]
    p = [v[r] for r in rot]
    # quad face (p1, p2, p5, p4) is the one not touching p0: pick its diagonal
    if min(p[1], p[5]) < min(p[2], p[4]):
        tets = [(p[0], p[1], p[2], p[5]), (p[0], p[1], p[5], p[4]), (p[0], p[4], p[5], p[3])]
    else:
        tets = [(p[0], p[1], p[2], p[4]), (p[0], p[4], p[2], p[5]), (p[0], p[4], p[5], p[3])]
    return tets


def _orient_tet(VX, t):
    a, b, c, d = t
    vol = np.dot(np.cross(VX[b] - VX[a], VX[c] - VX[a]), VX[d] - VX[a])
    return (a, c, b, d) if vol < 0 else (a, b, c, d)


def hybrid_mesh(ntri_side: int, n_wedge_layers: int, n_tet_layers: int,
                amp_frac: float = 0.2, seed0: int = 2000) -> Mesh:
    """Bottom `n_wedge_layers` layers of bumpy wedges (interfaces as in
    bumpy_layered_mesh, seeds seed0+k) under `n_tet_layers` flat layers whose
    prisms are each split into 3 tetrahedra by global vertex order.  The
    wedge/tet interface is conforming on triangle faces.  Element order:
    all wedges (column-major) first, then all tets."""
    L = n_wedge_layers + n_tet_layers
    bumps = {k: _bump_field(seed0 + k) for k in range(1, n_wedge_layers)}

    def iface(k, x, y):
        z = np.full_like(x, k / L, dtype=np.float64)
        if 0 < k < n_wedge_layers:
            z = z + amp_frac / L * bumps[k](x, y)
        return z
    full = layered_wedge_mesh(ntri_side, ntri_side, L, iface)
    VX = full.VX
    EToV_w = []
    EToV_t = []
    for e in range(full.K):
        layer = e % L
        if layer < n_wedge_layers:
            EToV_w.append(full.EToV[e])
        else:
            for t in _prism_to_tets(full.EToV[e]):
                t = _orient_tet(VX, t)
                EToV_t.append(list(t) + [-1, -1])
    EToV = np.vstack([np.asarray(EToV_w, dtype=np.int64).reshape(-1, 6),
                      np.asarray(EToV_t, dtype=np.int64).reshape(-1, 6)])
    etype = np.concatenate([np.full(len(EToV_w), WEDGE, dtype=np.uint8),
                            np.full(len(EToV_t), TET, dtype=np.uint8)])
    return Mesh(VX, EToV, etype, name=f"hybrid_{ntri_side}x{ntri_side}_{n_wedge_layers}w{n_tet_layers}t",
                meta=dict(nwedge=len(EToV_w), ntet=len(EToV_t)))


def tet_box_mesh(m: int, nlayers: int, box=(-1.0, 1.0, -1.0, 1.0), zrange=(-1.0, 1.0)) -> Mesh:
    """All-tetrahedral mesh: a flat layered prism mesh of the box with every
    prism split into 3 tets by global vertex order."""
    z0, z1 = zrange
    base = layered_wedge_mesh(m, m, nlayers, lambda k, x, y: np.full_like(x, z0 + (z1 - z0) * k / nlayers),
                              box=box)
    EToV_t = []
    for e in range(base.K):
        for t in _prism_to_tets(base.EToV[e]):
            EToV_t.append(list(_orient_tet(base.VX, t)) + [-1, -1])
    EToV = np.asarray(EToV_t, dtype=np.int64)
    return Mesh(base.VX, EToV, np.full(EToV.shape[0], TET, dtype=np.uint8),
                name=f"tetbox_{m}x{m}x{nlayers}")


# ----------------------------------------------------------------------------
# materials and fields
# ----------------------------------------------------------------------------

def uniform_material(K: int, c2: float = 1.0, rho: float = 1.0):
    return np.full(K, c2), np.full(K, rho)


def layered_wavespeed(mesh: Mesh, speeds=(2.5, 2.0, 1.5, 1.0)):
    """c by depth quartile of the layer index (bottom -> top), rho = 1."""
    L = mesh.meta["nlayers"]
    layer = np.arange(mesh.K) % L
    q = np.minimum(layer * len(speeds) // L, len(speeds) - 1)
    c = np.asarray(speeds)[q]
    return c * c, np.ones(mesh.K)


def random_material(K: int, seed: int, cmin: float = 1.0, cmax: float = 3.0,
                    rho_min: float = 1.0, rho_max: float = 1.0):
    rng = np.random.default_rng(seed)
    c = rng.uniform(cmin, cmax, size=K)
    rho = rng.uniform(rho_min, rho_max, size=K) if rho_max > rho_min else np.full(K, rho_min)
    return c * c, rho


def random_fields(total_nodes: int, seed: int, dtype=np.float64):
    """Seeded state in the canonical [4][total_nodes] layout, entries U(-1,1)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(4, total_nodes)).astype(dtype)


def gaussian_pulse(xyz: np.ndarray, center=(0.5, 0.5, 0.5), width: float = 0.05):
    """p0 = exp(-|x - xc|^2 / width^2), u0 = 0, at node coordinates xyz[3][n]."""
    r2 = sum((xyz[d] - center[d]) ** 2 for d in range(3))
    q = np.zeros((4, xyz.shape[1]))
    q[0] = np.exp(-r2 / width ** 2)
    return q


def standing_mode_unit_cube(xyz: np.ndarray, t: float):
    """Rigid-wall standing mode on [0,1]^3 with c = rho = 1:
    p = cos(pi x)cos(pi y)cos(pi z)cos(sqrt3 pi t),
    u = (sin cos cos, cos sin cos, cos cos sin) * sin(sqrt3 pi t)/sqrt3."""
    x, y, z = xyz
    w = math.sqrt(3.0) * math.pi
    cx, cy, cz = np.cos(np.pi * x), np.cos(np.pi * y), np.cos(np.pi * z)
    sx, sy, sz = np.sin(np.pi * x), np.sin(np.pi * y), np.sin(np.pi * z)
    st = math.sin(w * t) / math.sqrt(3.0)
    return np.stack([cx * cy * cz * math.cos(w * t), sx * cy * cz * st,
                     cx * sy * cz * st, cx * cy * sz * st])


def standing_mode_biunit_cube(xyz: np.ndarray, t: float):
    """Homogeneous-Dirichlet standing mode on [-1,1]^3 with c = rho = 1
    (Section 6.1): p = cos(pi x/2)cos(pi y/2)cos(pi z/2)cos(sqrt3 pi t/2)."""
    x, y, z = xyz
    h = 0.5 * np.pi
    w = math.sqrt(3.0) * h
    cx, cy, cz = np.cos(h * x), np.cos(h * y), np.cos(h * z)
    sx, sy, sz = np.sin(h * x), np.sin(h * y), np.sin(h * z)
    st = math.sin(w * t) / math.sqrt(3.0)
    return np.stack([cx * cy * cz * math.cos(w * t), sx * cy * cz * st,
                     cx * sy * cz * st, cx * cy * sz * st])


def merge_meshes(meshes, shift=(2.0, 0.0, 0.0)) -> Mesh:
    """Disjoint union of meshes (many small meshes advanced in one launch):
    vertex lists concatenated, mesh i translated by i * shift so the pieces do
    not touch, element lists concatenated in order.  Returns the merged mesh;
    meta["offsets"] holds each piece's first element."""
    VX, EToV, etype, offs = [], [], [], []
    nv = 0
    ne = 0
    for i, m in enumerate(meshes):
        VX.append(m.VX + np.asarray(shift, dtype=np.float64) * i)
        E = m.EToV.copy()
        E[E >= 0] += nv
        EToV.append(E)
        etype.append(m.etype)
        offs.append(ne)
        nv += m.VX.shape[0]
        ne += m.K
    return Mesh(np.vstack(VX), np.vstack(EToV), np.concatenate(etype), name="merged", meta={"offsets": offs})


def layer_major(mesh: Mesh, nlayers: int) -> tuple:
    """The same column-major layered mesh (element k = column * nlayers + layer)
    listed layer by layer instead, so that no vertical neighbour shares a
    32-element block: the reference order for measuring what the column order
    saves.  Returns (mesh, perm) with new element i = old element perm[i]."""
    k = np.arange(mesh.EToV.shape[0])
    perm = np.lexsort((k // nlayers, k % nlayers))
    return Mesh(mesh.VX, mesh.EToV[perm], mesh.etype[perm], mesh.name + "_layer_major", dict(mesh.meta)), perm


def surface_shots(nshots: int, seed: int, depth: float = 0.01, margin: float = 0.05):
    """Seeded source positions just below the top surface z = 1 of [0,1]^3."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(margin, 1.0 - margin, size=(nshots, 2))
    return [(float(x), float(y), 1.0 - depth) for x, y in xy]


def inclusion_model(mesh: Mesh, amp: float = 0.5, center=(0.5, 0.5, 0.9), width: float = 0.2,
                    c2_top: float = 1.0, c2_bottom: float = 2.25, z_interface: float = 0.5):
    """Per-element c^2 of a two-layer model (c2_bottom below z_interface, c2_top
    above, by element centroid) plus a smooth Gaussian inclusion of amplitude
    `amp`; rho = 1.  Returns (c2, rho).  The default inclusion sits just below
    the surface: the surface sources' wavefield crosses it within the 800
    steps of the differentiation workload (t = 0.12), so the misfit between
    the two models' traces is a real signal (0.3% of the trace norm); an
    inclusion at mid-depth would not be reached, and the traces of the two
    models would differ by less than FP32 rounding."""
    V = mesh.VX[np.where(mesh.EToV >= 0, mesh.EToV, mesh.EToV[:, :1])]
    nv = np.where(mesh.etype == WEDGE, 6, 4)[:, None]
    cen = np.array([(V[k, :nv[k, 0]]).mean(axis=0) for k in range(mesh.K)])
    c2 = np.where(cen[:, 2] < z_interface, c2_bottom, c2_top)
    r2 = ((cen - np.asarray(center)) ** 2).sum(axis=1)
    c2 = c2 + amp * np.exp(-r2 / width ** 2)
    return c2, np.ones(mesh.K)


def surface_receivers(n_side: int, depth: float = 0.01, margin: float = 0.05):
    """n_side x n_side grid of receiver points just below the top surface z = 1."""
    g = np.linspace(margin, 1.0 - margin, n_side)
    return [(float(x), float(y), 1.0 - depth) for y in g for x in g]
