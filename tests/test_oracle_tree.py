"""Pins for oracle.tree (clustering and one-box-buffer lists, Section 3)."""
import numpy as np
import pytest

import pie_inputs as pi
from oracle.mesh import build_topology
from oracle.tree import build_tree, offset_code
from oracle.asd import far_offsets


@pytest.mark.parametrize("n,L", [(2, 3), (2, 4), (3, 4), (3, 5)])
def test_pairs_partitioned_once(n, L):
    """Every ordered triangle pair is near at the leaves or in exactly one
    interaction list at exactly one level."""
    xyz, tri = pi.icosphere(n)
    top = build_topology(xyz, tri)
    tr = build_tree(top.centroid, top.xyz, L, side=2.0)
    T = top.T
    leaf_of = np.repeat(np.arange(tr.keys[L].size), np.diff(tr.leaf_start))  # tree order
    count = np.zeros((T, T), np.int64)
    nb = np.diff(tr.leaf_start)
    for b in range(tr.keys[L].size):
        for q in tr.near_idx[tr.near_ptr[b]:tr.near_ptr[b + 1]]:
            count[tr.leaf_start[b]:tr.leaf_start[b + 1], tr.leaf_start[q]:tr.leaf_start[q + 1]] += 1
    for l in range(3, L + 1):
        # box of each tree-ordered triangle at level l
        box_l = np.searchsorted(tr.keys[l], tr.leaf_key_of_tri >> (3 * (L - l)))
        for d in range(tr.keys[l].size):
            td = np.nonzero(box_l == d)[0]
            for s in tr.il_idx[l][tr.il_ptr[l][d]:tr.il_ptr[l][d + 1]]:
                ts = np.nonzero(box_l == s)[0]
                count[np.ix_(td, ts)] += 1
    assert np.all(count == 1)
    assert nb.sum() == T


def test_list_sizes_symmetry_and_offsets():
    xyz, tri = pi.icosphere(4)
    top = build_topology(xyz, tri)
    L = 5
    tr = build_tree(top.centroid, top.xyz, L, side=2.0)
    assert np.max(np.diff(tr.near_ptr)) <= 27
    pairs = {(b, q) for b in range(tr.keys[L].size) for q in tr.near_idx[tr.near_ptr[b]:tr.near_ptr[b + 1]]}
    assert all((q, b) in pairs for b, q in pairs)
    offs = far_offsets()
    for l in range(3, L + 1):
        assert np.max(np.diff(tr.il_ptr[l])) <= 189
        ptr, idx, off = tr.il_ptr[l], tr.il_idx[l], tr.il_off[l]
        lists = {d: set(idx[ptr[d]:ptr[d + 1]]) for d in range(tr.keys[l].size)}
        for d, ss in lists.items():
            for s in ss:
                assert d in lists[s]
        for d in range(tr.keys[l].size):
            for j in range(ptr[d], ptr[d + 1]):
                assert np.array_equal(offs[off[j]], tr.ijk[l][d] - tr.ijk[l][idx[j]])


def test_offset_code_order():
    offs = far_offsets()
    for i, o in enumerate(offs):
        assert offset_code(tuple(o)) == i
    assert offset_code((1, -1, 0)) == -1


def test_leaf_index_formula_and_order():
    xyz, tri = pi.icosphere(3)
    top = build_topology(xyz, tri)
    tr = build_tree(top.centroid, top.xyz, 4, side=2.0)
    # tree order sorted by (key, triangle index)
    k = tr.leaf_key_of_tri
    assert np.all((np.diff(k) > 0) | ((np.diff(k) == 0) & (np.diff(tr.perm) > 0)))
    # brute-force box membership: centroid inside the half-open leaf cube
    a = tr.box_size(4)
    boxes = np.searchsorted(tr.keys[4], k)
    lo = tr.x0 + tr.ijk[4][boxes] * a
    c = top.centroid[tr.perm]
    assert np.all(c >= lo - 1e-12) and np.all(c < lo + a + 1e-12)


def test_cube_faces_on_box_planes():
    """Cube faces lie exactly on the root's boundary planes and, with a grid
    aligned to the boxes, centroids fall on interior planes' sides only through
    the half-open rule and the clamp; every pair is still partitioned once."""
    xyz, tri = pi.cube(8)
    top = build_topology(xyz, tri)
    tr = build_tree(top.centroid, top.xyz, 4, side=1.0)
    a = tr.box_size(4)
    k = tr.leaf_key_of_tri
    boxes = np.searchsorted(tr.keys[4], k)
    lo = tr.x0 + tr.ijk[4][boxes] * a
    c = top.centroid[tr.perm]
    inside = (c >= lo) & ((c < lo + a) | (np.isclose(c, 0.5) & np.isclose(lo + a, 0.5)))
    assert np.all(inside)
