"""Cubic-box oct-tree and one-box-buffer lists (Section 3: "standard
clustering by enclosing the object in a cubic box and recursively dividing it
into subboxes", "one-box-buffer scheme").

Readings:
* level 1 is the root box; three levels means translations at one level
  (Section 4), so translations happen at levels 3..L;
* triangles are clustered by centroid; the root cube is centred on the vertex
  bounding-box centre, its side is the largest bounding-box extent unless given;
* leaf index per axis = clamp(floor((c - x0) * (2^(L-1) / side)), 0, 2^(L-1)-1)
  in IEEE double (one subtraction, one multiplication, no fused multiply-add);
* Morton key: bit b of the x / y / z index goes to bit 3b+2 / 3b+1 / 3b; a box's
  key at level l is the leaf key shifted right by 3 (L - l); triangles are
  ordered by (leaf key, triangle index);
* near list of a leaf box: leaf boxes whose indices differ by at most 1 on
  every axis (itself included); interaction list of a box at level l >= 3:
  children of its parent's neighbours (parent included) that are not its own
  neighbours.  Lists are sorted by box number.

Integer output, compared bit-exactly with the CUDA library.  Pinned in
tests/test_oracle_tree.py (every triangle pair is near at the leaves or far at
exactly one level; list sizes <= 27 and <= 189; near lists symmetric; brute
force membership on small meshes).
"""
from dataclasses import dataclass, field

import numpy as np


def morton(ix, iy, iz, bits):
    key = np.zeros(np.shape(ix), np.int64)
    for b in range(bits):
        key |= ((ix >> b) & 1) << (3 * b + 2)
        key |= ((iy >> b) & 1) << (3 * b + 1)
        key |= ((iz >> b) & 1) << (3 * b)
    return key


def demorton(key, bits):
    ix = np.zeros(np.shape(key), np.int64)
    iy = np.zeros_like(ix)
    iz = np.zeros_like(ix)
    for b in range(bits):
        ix |= ((key >> (3 * b + 2)) & 1) << b
        iy |= ((key >> (3 * b + 1)) & 1) << b
        iz |= ((key >> (3 * b)) & 1) << b
    return ix, iy, iz


def root_box(xyz, side=0.0):
    lo = xyz.min(axis=0)
    hi = xyz.max(axis=0)
    center = (lo + hi) * 0.5
    if side <= 0:
        side = float(np.max(hi - lo))
    return center, side


@dataclass
class Tree:
    L: int
    center: np.ndarray
    side: float
    x0: np.ndarray
    perm: np.ndarray                     # tree order -> mesh triangle
    leaf_key_of_tri: np.ndarray          # per tree-ordered triangle
    keys: dict = field(default_factory=dict)       # level -> sorted box keys
    ijk: dict = field(default_factory=dict)        # level -> [nb,3] box indices
    parent: dict = field(default_factory=dict)     # level -> parent box number
    leaf_start: np.ndarray = None        # [nleaf+1] triangle ranges (tree order)
    near_ptr: np.ndarray = None
    near_idx: np.ndarray = None
    il_ptr: dict = field(default_factory=dict)     # level -> CSR pointer
    il_idx: dict = field(default_factory=dict)     # level -> source box numbers
    il_off: dict = field(default_factory=dict)     # level -> offset code 0..315

    def box_size(self, l):
        return self.side / (1 << (l - 1))

    def box_centers(self, l):
        return self.x0 + (self.ijk[l] + 0.5) * self.box_size(l)


def offset_code(d):
    """Index of an offset in oracle.asd.far_offsets order, -1 if near."""
    dx, dy, dz = d
    if max(abs(dx), abs(dy), abs(dz)) <= 1:
        return -1
    full = (dx + 3) * 49 + (dy + 3) * 7 + (dz + 3)
    # number of near offsets (|.|inf <= 1) with smaller full code
    inner_before = 0
    for ex in range(-1, 2):
        for ey in range(-1, 2):
            for ez in range(-1, 2):
                if (ex + 3) * 49 + (ey + 3) * 7 + (ez + 3) < full:
                    inner_before += 1
    return full - inner_before


def build_tree(centroids, xyz, L, side=0.0) -> Tree:
    centroids = np.asarray(centroids, np.float64)
    center, side = root_box(np.asarray(xyz, np.float64), side)
    x0 = center - side * 0.5
    nleaf = 1 << (L - 1)
    scale = nleaf / side
    idx = np.floor((centroids - x0) * scale).astype(np.int64)
    idx = np.clip(idx, 0, nleaf - 1)
    key = morton(idx[:, 0], idx[:, 1], idx[:, 2], L - 1)
    perm = np.lexsort((np.arange(len(key)), key))
    tr = Tree(L=L, center=center, side=side, x0=x0, perm=perm, leaf_key_of_tri=key[perm])
    for l in range(1, L + 1):
        k = np.unique(tr.leaf_key_of_tri >> (3 * (L - l)))
        tr.keys[l] = k
        ix, iy, iz = demorton(k, l - 1)
        tr.ijk[l] = np.stack([ix, iy, iz], axis=1)
        if l > 1:
            tr.parent[l] = np.searchsorted(tr.keys[l - 1], k >> 3)
    lk = tr.keys[L]
    tr.leaf_start = np.searchsorted(tr.leaf_key_of_tri, lk, side="left")
    tr.leaf_start = np.append(tr.leaf_start, len(key)).astype(np.int64)

    def lookup(l):
        return {tuple(v): i for i, v in enumerate(tr.ijk[l])}

    # near lists at the leaves
    look = lookup(L)
    ptr, lst = [0], []
    for b, v in enumerate(tr.ijk[L]):
        nb = []
        for d in np.ndindex(3, 3, 3):
            q = tuple(v + np.array(d) - 1)
            if q in look:
                nb.append(look[q])
        lst += sorted(nb)
        ptr.append(len(lst))
    tr.near_ptr = np.array(ptr, np.int64)
    tr.near_idx = np.array(lst, np.int64)

    # interaction lists, levels 3..L
    for l in range(3, L + 1):
        look_l = lookup(l)
        ptr, lst, off = [0], [], []
        for b, v in enumerate(tr.ijk[l]):
            pv = v >> 1
            cand = []
            for d in np.ndindex(3, 3, 3):
                q = pv + np.array(d) - 1
                for o in np.ndindex(2, 2, 2):
                    c = tuple(2 * q + np.array(o))
                    if c in look_l:
                        dd = v - np.array(c)
                        if np.max(np.abs(dd)) > 1:
                            cand.append(look_l[c])
            cand = sorted(cand)
            lst += cand
            off += [offset_code(tuple(v - tr.ijk[l][c])) for c in cand]
            ptr.append(len(lst))
        tr.il_ptr[l] = np.array(ptr, np.int64)
        tr.il_idx[l] = np.array(lst, np.int64)
        tr.il_off[l] = np.array(off, np.int64)
    return tr
