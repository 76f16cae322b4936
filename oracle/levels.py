"""Split of the PIE product by the oct-tree level that carries each
interaction (Section 3), for the error of the far part level by level.

TEST INFRASTRUCTURE: imported only by tests/, never by the library.

Reading (the paper states the one-box-buffer rule of the MLFMA, not this
split in words): triangles sit in boxes by centroid; two boxes of one level
are neighbours when their integer indices differ by at most one in every
coordinate.  A triangle pair (t, s) is near -- level 0 -- when its leaf boxes
are neighbours.  Otherwise the MLFMA translates it at exactly one level: the
coarsest level l >= 3 at which its two boxes are not neighbours (their
parents are: at level 2 all eight boxes are neighbours), which is the level
at which the source box sits in the destination box's interaction list.
Hence Z = Z_near + sum_{l=3..L} Z_l exactly, where Z_l keeps the pairs of
level l, and oracle.dense.assemble / rows with pair_mask = mask(l) give each
part.

Pinned in tests/test_oracle_levels.py: the classes against the near lists
and interaction lists that oracle.tree builds by its own route, symmetry of
the classes, and the parts summing to the dense matrix.
"""
import numpy as np

from .tree import build_tree


class PairLevels:
    """Level of triangle pairs (mesh-order triangle indices) in the tree of
    depth L over the given centroids (root box as in oracle.tree)."""

    def __init__(self, centroids, xyz, L, side=0.0):
        tr = build_tree(centroids, xyz, L, side)
        self.L = L
        self.tree = tr
        tri_box = np.repeat(np.arange(tr.keys[L].size), np.diff(tr.leaf_start))   # tree order
        inv = np.empty_like(tr.perm)
        inv[tr.perm] = np.arange(tr.perm.size)
        self.ijk = tr.ijk[L][tri_box[inv]]                                        # [T,3], mesh order

    def level(self, t, s):
        """0 for near pairs, else the level l in [3, L] that translates them."""
        a = self.ijk[t]
        b = self.ijk[s]
        lev = np.zeros(np.broadcast_shapes(np.shape(t), np.shape(s)), np.int64)
        for l in range(self.L, 2, -1):
            sh = self.L - l
            far = np.max(np.abs((a >> sh) - (b >> sh)), axis=-1) > 1
            lev = np.where(far, l, lev)
        return lev

    def mask(self, l):
        """pair_mask for oracle.dense keeping the pairs of level l."""
        return lambda t, s: self.level(t, s) == l
