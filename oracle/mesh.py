"""Oracle connectivity: node coordinates, face matching and face-node maps.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Global node numbering is canonical: element by element in input order, each
element's nodes contiguous in its reference order (wedge n = j*Nt + i).
Faces are matched by their vertex sets; face nodes are matched to the
neighbour's face nodes by physical coordinates (nearest point), which needs
no orientation bookkeeping at all.
"""
from __future__ import annotations

import numpy as np

from . import reference as R

WEDGE = 6
TET = 4

# reference faces as local vertex lists
WEDGE_FACE_VERTS = ((0, 1, 2), (3, 4, 5), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5))
TET_FACE_VERTS = R.Tet.FACE_VERTS


class Connectivity:
    def __init__(self, VX, EToV, etype, N: int):
        self.VX = np.asarray(VX, dtype=np.float64)
        self.EToV = np.asarray(EToV, dtype=np.int64)
        self.etype = np.asarray(etype, dtype=np.uint8)
        self.N = N
        self.K = self.EToV.shape[0]
        self.W = R.wedge(N)
        self.T = R.tet(N)
        self.Np = np.where(self.etype == WEDGE, self.W.Np, self.T.Np)
        self.offset = np.concatenate([[0], np.cumsum(self.Np)])
        self.total_nodes = int(self.offset[-1])
        self.wedges = np.nonzero(self.etype == WEDGE)[0]
        self.tets = np.nonzero(self.etype == TET)[0]

        # node coordinates via the vertex maps
        self.xyz = np.zeros((3, self.total_nodes))
        vw, _ = R.wedge_vertex_functions(self.W.x)
        vt, _ = R.tet_vertex_functions(self.T.x)
        for k in range(self.K):
            if self.etype[k] == WEDGE:
                X = vw @ self.VX[self.EToV[k, :6]]
            else:
                X = vt @ self.VX[self.EToV[k, :4]]
            self.xyz[:, self.offset[k]:self.offset[k + 1]] = X.T

        # face matching by vertex sets
        table = {}
        self.EToE = np.full((self.K, 5), -1, dtype=np.int64)
        self.EToF = np.full((self.K, 5), -1, dtype=np.int64)
        for k in range(self.K):
            for f, fv in enumerate(self.face_verts(k)):
                key = tuple(sorted(int(self.EToV[k, v]) for v in fv))
                if key in table:
                    k2, f2 = table.pop(key)
                    self.EToE[k, f], self.EToF[k, f] = k2, f2
                    self.EToE[k2, f2], self.EToF[k2, f2] = k, f
                else:
                    table[key] = (k, f)
        # remaining entries are boundary faces

        # face-node maps: for each (k, f) the global ids of own face nodes
        # (vmapM) and of the coincident neighbour nodes (vmapP; own for boundary)
        self.vmapM = {}
        self.vmapP = {}
        for k in range(self.K):
            for f in range(self.nfaces(k)):
                gM = self.offset[k] + self.face_nodes(k, f)
                self.vmapM[(k, f)] = gM
                k2 = self.EToE[k, f]
                if k2 < 0:
                    self.vmapP[(k, f)] = gM.copy()
                    continue
                f2 = self.EToF[k, f]
                gP_all = self.offset[k2] + self.face_nodes(k2, f2)
                XM = self.xyz[:, gM].T
                XP = self.xyz[:, gP_all].T
                d = np.linalg.norm(XM[:, None, :] - XP[None, :, :], axis=2)
                m = np.argmin(d, axis=1)
                scale = np.max(np.ptp(XM, axis=0)) + 1e-300
                if np.max(d[np.arange(len(m)), m]) > 1e-8 * scale or len(set(m.tolist())) != len(m):
                    raise ValueError(f"face nodes of element {k} face {f} do not match neighbour {k2}")
                self.vmapP[(k, f)] = gP_all[m]

    def nfaces(self, k: int) -> int:
        return 5 if self.etype[k] == WEDGE else 4

    def face_verts(self, k: int):
        return WEDGE_FACE_VERTS if self.etype[k] == WEDGE else TET_FACE_VERTS

    def face_nodes(self, k: int, f: int) -> np.ndarray:
        return self.W.faces[f] if self.etype[k] == WEDGE else self.T.faces[f]
