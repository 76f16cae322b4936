"""The other shapes of the batched configuration: cube (faces on box planes),
2:1:1 ellipsoid, capped cylinder.  Tree and lists bit-exact at the full
configuration sizes; the product within 1e-3 of the dense oracle on small
versions (kR = 0.01)."""
import numpy as np
import pytest

import pie_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    return pg


@pytest.mark.parametrize("name,mesh,L,side", [
    ("cube", lambda: pi.cube(32), 5, 1.0),
    ("ellipsoid", lambda: pi.octasphere(6, (1.0, 0.5, 0.5)), 6, 0.0),
    ("cylinder", lambda: pi.cylinder(), 6, 0.0),
])
def test_tree_bit_exact_full_size(pg, name, mesh, L, side):
    from oracle.mesh import build_topology
    from oracle.tree import build_tree
    xyz, tri = mesh()
    pr = pg.Problem(pg.Mesh(xyz, tri), 0.01, L, root_side=side, precision=pg.PIE_MIXED)
    top = build_topology(xyz, tri)
    tr = build_tree(top.centroid, top.xyz, L, side=side)
    assert np.array_equal(pr.perm(), tr.perm)
    for l in range(1, L + 1):
        keys, ptr, idx, off = pr.level(l)
        assert np.array_equal(keys, tr.keys[l])
        if l >= 3:
            assert np.array_equal(ptr, tr.il_ptr[l]) and np.array_equal(idx, tr.il_idx[l])
            assert np.array_equal(off, tr.il_off[l])
    ptr, idx = pr.near()
    assert np.array_equal(ptr, tr.near_ptr) and np.array_equal(idx, tr.near_idx)


@pytest.mark.parametrize("name,mesh,side", [
    ("cube", lambda: pi.cube(8), 1.0),
    ("ellipsoid", lambda: pi.octasphere(3, (1.0, 0.5, 0.5)), 0.0),
    ("cylinder", lambda: pi.cylinder(nseg=16, nrings=2, nrows=8), 0.0),
])
def test_product_matches_dense_small(pg, name, mesh, side):
    import torch
    from oracle.dense import assemble
    from oracle.mesh import build_topology
    xyz, tri = mesh()
    k = 0.01
    top = build_topology(xyz, tri)
    Z = assemble(top, k)
    pr = pg.Problem(pg.Mesh(xyz, tri), k, 3, root_side=side, precision=pg.PIE_MIXED)
    E, T = pr.E, pr.T
    for x in (np.r_[pi.complex_normal(E, 1), np.zeros(T)], np.r_[np.zeros(E), pi.complex_normal(T, 2)]):
        y = pr.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        yd = Z @ x
        for sl in (slice(0, E), slice(E, None)):
            err = np.linalg.norm(y[sl] - yd[sl]) / np.linalg.norm(yd[sl])
            assert err < 1e-3, (name, err)
