"""The product split by tree level (pie_apply_levels) against the exact
level parts of the dense oracle (oracle.levels): the Eq. (4)-(5) error of
the far part, level by level.  Small mesh: every level against the dense
part matrices, the parts summing to the product.  The 6-level, 81,920-
triangle sphere at kR = 1e-3: sampled rows of each level's part against the
oracle's row sums over that level's pairs."""
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


@pytest.mark.parametrize("prec", [0, 2])
def test_levels_small_vs_dense_parts(pg, prec):
    import torch
    from oracle.dense import assemble
    from oracle.levels import PairLevels
    from oracle.mesh import build_topology
    k, L = 0.01, 4
    xyz, tri = pi.icosphere(3)
    top = build_topology(xyz, tri)
    pl = PairLevels(top.centroid, top.xyz, L, side=2.0)
    pr = pg.Problem(pg.Mesh(xyz, tri), k, L, root_side=2.0, precision=prec)
    E = top.E
    Z = assemble(top, k)
    for x in (np.r_[pi.complex_normal(E, 1), np.zeros(top.T)], np.r_[np.zeros(E), pi.complex_normal(top.T, 2)]):
        xd = torch.from_numpy(x).cuda()
        y = Z @ x
        total = pr.apply_levels(xd, [], near=True).cpu().numpy()
        yn = assemble(top, k, pair_mask=pl.mask(0)) @ x
        tol_near = 1e-12 if prec == 0 else 1e-6
        assert np.linalg.norm(total - yn) <= tol_near * np.linalg.norm(yn)
        for l in (3, 4):
            yl = pr.apply_levels(xd, [l]).cpu().numpy()
            total = total + yl
            yd = assemble(top, k, pair_mask=pl.mask(l)) @ x
            for sl in (slice(0, E), slice(E, None)):
                d = np.linalg.norm(yl[sl] - yd[sl])
                assert d < 1e-3 * np.linalg.norm(y[sl]), (l, d / np.linalg.norm(y[sl]))
        full = pr.apply(xd).cpu().numpy()
        assert np.linalg.norm(total - full) <= 1e-6 * np.linalg.norm(full)


def test_levels_config2_sampled_rows(pg):
    """81,920 triangles, L = 6, kR = 1e-3 (FP64 far part): per level l = 3..6
    the relative error of the level part on 8 sampled rows (4 RWG, 4 pulse),
    against the product's size on those rows."""
    import torch
    from oracle.dense import rows
    from oracle.levels import PairLevels
    from oracle.mesh import build_topology
    k, L = 1e-3, 6
    xyz, tri = pi.icosphere(6)
    top = build_topology(xyz, tri)
    pl = PairLevels(top.centroid, top.xyz, L, side=2.0)
    pr = pg.Problem(pg.Mesh(xyz, tri), k, L, root_side=2.0, precision=pg.PIE_MIXED)
    x = pi.complex_normal(top.N, 77)
    xd = torch.from_numpy(x).cuda()
    rng = np.random.default_rng(5)
    which = np.r_[rng.choice(top.E, 4, replace=False), top.E + rng.choice(top.T, 4, replace=False)]
    full = pr.apply(xd).cpu().numpy()[which]
    errs = {}
    for l in range(3, L + 1):
        yl = pr.apply_levels(xd, [l]).cpu().numpy()[which]
        yd = np.array(rows(top, k, which, x, pair_mask=pl.mask(l)))
        for name, sl in (("rwg", slice(0, 4)), ("pulse", slice(4, 8))):
            errs[(l, name)] = np.linalg.norm(yl[sl] - yd[sl]) / np.linalg.norm(full[sl])
    print("per-level error (relative to the product on the sampled rows):",
          {f"{l}/{n}": f"{e:.2e}" for (l, n), e in errs.items()})
    assert max(errs.values()) < 1e-3, errs
