"""Pins for oracle.levels: the split of the product by tree level.

The pair classes are checked against the near lists and interaction lists
that oracle.tree builds by its own route (box lookups, not index
arithmetic), the parts of the dense matrix must sum to it, and the CPU MLFMA
restricted to one level's translations must approximate that level's part
of the dense product to the product tolerance."""
import numpy as np
import pytest

import pie_inputs as pi
from oracle.dense import assemble
from oracle.levels import PairLevels
from oracle.mesh import build_topology
from oracle.mlfma import MLFMA

K = 0.01


@pytest.fixture(scope="module")
def sphere2():
    xyz, tri = pi.icosphere(2)
    top = build_topology(xyz, tri)
    return xyz, tri, top


def test_classes_match_tree_lists(sphere2):
    xyz, tri, top = sphere2
    L = 4
    pl = PairLevels(top.centroid, top.xyz, L, side=2.0)
    tr = pl.tree
    T = top.T
    t, s = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    lev = pl.level(t.ravel(), s.ravel()).reshape(T, T)
    assert np.array_equal(lev, lev.T)
    assert set(np.unique(lev)) <= {0, 3, 4}
    # box number of every mesh triangle at every level, from the tree's keys
    key_of = np.empty(T, np.int64)
    key_of[tr.perm] = tr.leaf_key_of_tri

    def box(l, tri_idx):
        return np.searchsorted(tr.keys[l], key_of[tri_idx] >> (3 * (L - l)))

    want = np.full((T, T), -1, np.int64)
    bL = box(L, np.arange(T))
    for b in range(tr.keys[L].size):
        nb = tr.near_idx[tr.near_ptr[b]:tr.near_ptr[b + 1]]
        rows = np.nonzero(bL == b)[0]
        cols = np.nonzero(np.isin(bL, nb))[0]
        want[np.ix_(rows, cols)] = 0
    for l in range(3, L + 1):
        bl = box(l, np.arange(T))
        for b in range(tr.keys[l].size):
            il = tr.il_idx[l][tr.il_ptr[l][b]:tr.il_ptr[l][b + 1]]
            rows = np.nonzero(bl == b)[0]
            cols = np.nonzero(np.isin(bl, il))[0]
            assert np.all(want[np.ix_(rows, cols)] == -1)      # no pair in two classes
            want[np.ix_(rows, cols)] = l
    assert np.all(want >= 0)                                    # every pair in one class
    assert np.array_equal(lev, want)


def test_parts_sum_to_dense(sphere2):
    xyz, tri, top = sphere2
    pl = PairLevels(top.centroid, top.xyz, 4, side=2.0)
    Z = assemble(top, K)
    parts = {l: assemble(top, K, pair_mask=pl.mask(l)) for l in (0, 3, 4)}
    S = sum(parts.values())
    assert np.max(np.abs(S - Z)) <= 1e-13 * np.max(np.abs(Z))
    for l, Zl in parts.items():
        assert np.max(np.abs(Zl - Zl.T)) <= 1e-13 * np.max(np.abs(Z))   # each part complex symmetric
        assert np.count_nonzero(Zl) > 0, l


def test_mlfma_per_level_error():
    """The CPU MLFMA with one level's translations alone against that level's
    exact part: the Eq. (4)-(5) error holds level by level (kappa_l a_l is
    the same at every level)."""
    xyz, tri = pi.icosphere(3)
    top = build_topology(xyz, tri)
    L = 4
    pl = PairLevels(top.centroid, top.xyz, L, side=2.0)
    M = MLFMA(xyz, tri, K, L, side=2.0)
    E = top.E
    Z = assemble(top, K)
    parts = {l: assemble(top, K, pair_mask=pl.mask(l)) for l in (3, 4)}
    for x in (np.r_[pi.complex_normal(E, 1), np.zeros(top.T)], np.r_[np.zeros(E), pi.complex_normal(top.T, 2)]):
        y = Z @ x
        for l in (3, 4):
            yd = parts[l] @ x
            ym = M.apply(x, near=False, levels={l})
            for sl in (slice(0, E), slice(E, None)):
                # each level's error is a fraction of the product's 1e-3 budget
                # (measured 2.4e-4 .. 5.9e-4; 0.7e-3 .. 2.7e-3 of the level's own part)
                d = np.linalg.norm(ym[sl] - yd[sl])
                assert d < 1e-3 * np.linalg.norm(y[sl]), (l, d / np.linalg.norm(y[sl]))
                assert d < 5e-3 * np.linalg.norm(yd[sl]), (l, d / np.linalg.norm(yd[sl]))
    # the near part of the MLFMA is the near class exactly
    x = pi.complex_normal(top.N, 3)
    yn = M.apply(x, far=False)
    yd = assemble(top, K, pair_mask=pl.mask(0)) @ x
    assert np.linalg.norm(yn - yd) <= 1e-12 * np.linalg.norm(yd)
