"""Test helper: cut a face-connected patch out of a large mesh so the CPU
oracle can check sampled elements of a full-size GPU run.

A stage couples an element to its face neighbours only, so after s stages an
element depends on elements within s face hops.  An oracle run on the patch
of radius >= s around the sampled elements reproduces them exactly (patch
faces that are interior in the full mesh become spurious boundaries, but
their influence needs more than s stages to reach the centre)."""
import numpy as np

WEDGE_FACES = ((0, 1, 2, -1), (3, 4, 5, -1), (0, 1, 4, 3), (1, 2, 5, 4), (2, 0, 3, 5))
TET_FACES = ((0, 1, 2, -1), (0, 1, 3, -1), (1, 2, 3, -1), (0, 2, 3, -1))


def face_adjacency(EToV, etype):
    """(K, 5) neighbour element per face (-1 boundary), vectorised by sorting
    face vertex keys."""
    K = EToV.shape[0]
    keys, owner = [], []
    for f in range(5):
        for typ, faces in ((6, WEDGE_FACES), (4, TET_FACES)):
            if f >= len(faces):
                continue
            sel = np.nonzero(etype == typ)[0]
            if len(sel) == 0:
                continue
            fv = [v for v in faces[f] if v >= 0]
            k = np.sort(EToV[sel][:, fv], axis=1)
            if k.shape[1] == 3:
                k = np.column_stack([k, np.full(len(sel), -1)])
            keys.append(k)
            owner.append(np.column_stack([sel, np.full(len(sel), f)]))
    keys = np.vstack(keys)
    owner = np.vstack(owner)
    order = np.lexsort(keys.T[::-1])
    ks = keys[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    nbr = np.full((K, 5), -1, dtype=np.int64)
    i = np.nonzero(same)[0]
    a, b = owner[order[i]], owner[order[i + 1]]
    nbr[a[:, 0], a[:, 1]] = b[:, 0]
    nbr[b[:, 0], b[:, 1]] = a[:, 0]
    return nbr


def patch(nbr, seeds, radius):
    """Elements within `radius` face hops of the seeds (sorted)."""
    cur = np.unique(np.asarray(seeds))
    seen = set(cur.tolist())
    for _ in range(radius):
        nxt = nbr[cur].ravel()
        nxt = np.unique(nxt[nxt >= 0])
        new = [x for x in nxt.tolist() if x not in seen]
        seen.update(new)
        cur = np.asarray(new, dtype=np.int64)
        if len(cur) == 0:
            break
    return np.asarray(sorted(seen), dtype=np.int64)


def submesh(mesh_VX, EToV, etype, elems):
    """Sub-mesh of the given elements with compacted vertex numbering."""
    E = EToV[elems]
    used = np.unique(E[E >= 0])
    remap = -np.ones(mesh_VX.shape[0], dtype=np.int64)
    remap[used] = np.arange(len(used))
    E2 = np.where(E >= 0, remap[np.maximum(E, 0)], -1)
    return mesh_VX[used], E2, etype[elems]


def node_index(Np_of_elem, elems):
    """Canonical node ids of `elems` in the full mesh (per-element Np array)."""
    off = np.concatenate([[0], np.cumsum(Np_of_elem)])
    return np.concatenate([np.arange(off[k], off[k + 1]) for k in elems])
