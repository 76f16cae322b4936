"""Parity at full size, in the launch configuration bench.py times: the
819,200-unknown sphere (icosphere n = 7), kR = 1e-3, 7 levels,
x = complex normal with seed 1234, PIE_MIXED and then PIE_FP64.  Sampled
outputs are computed one by one by the oracle: full rows of the dense
product (bar 1e-3, the accuracy of the approximate diagonalization) and
near-part rows over the oracle's own tree (bar 1e-6 with float pair
moments, 1e-10 with double ones)."""
import numpy as np
import pytest

import pie_inputs as pi

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_bench_workload_sampled_rows():
    import torch

    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    from oracle.dense import rows
    from oracle.mesh import build_topology
    from oracle.tree import build_tree

    k = 1e-3
    xyz, tri = pi.icosphere(7)
    pr = pg.Problem(pg.Mesh(xyz, tri), k, 7, root_side=2.0, precision=pg.PIE_MIXED)
    x = pi.complex_normal(pr.N, 1234)
    xd = torch.from_numpy(x).cuda()
    y = pr.apply(xd).cpu().numpy()
    yn = pr.apply(xd, near_only=True).cpu().numpy()
    top = build_topology(xyz, tri)
    E = top.E
    rng = np.random.default_rng(77)
    which = np.r_[rng.choice(E, 5, replace=False), E + rng.choice(top.T, 5, replace=False)]
    yo = rows(top, k, which, x)
    for sl in (slice(0, 5), slice(5, 10)):
        assert np.linalg.norm(y[which][sl] - yo[sl]) <= 1e-3 * np.linalg.norm(yo[sl])
    tr = build_tree(top.centroid, top.xyz, 7, side=2.0)
    L = 7
    leaf = np.empty(top.T, np.int64)
    leaf[tr.perm] = np.repeat(np.arange(tr.keys[L].size), np.diff(tr.leaf_start))
    ijk = tr.ijk[L][leaf]

    def near(t, s):
        return np.max(np.abs(ijk[s] - ijk[t]), axis=1) <= 1

    yno = rows(top, k, which, x, pair_mask=near)
    for sl in (slice(0, 5), slice(5, 10)):
        assert np.linalg.norm(yn[which][sl] - yno[sl]) <= 1e-6 * np.linalg.norm(yno[sl])
    print("full-size sampled rows: far+near", np.linalg.norm(y[which] - yo) / np.linalg.norm(yo),
          "near", np.linalg.norm(yn[which] - yno) / np.linalg.norm(yno))
    # the plain FP64 form on the same rows: the same far part, the near part
    # in complex double (its pair integrals then match the oracle's to 1e-12)
    del pr
    torch.cuda.empty_cache()
    p64 = pg.Problem(pg.Mesh(xyz, tri), k, 7, root_side=2.0, precision=pg.PIE_FP64)
    y64 = p64.apply(xd).cpu().numpy()
    yn64 = p64.apply(xd, near_only=True).cpu().numpy()
    for sl in (slice(0, 5), slice(5, 10)):
        assert np.linalg.norm(y64[which][sl] - yo[sl]) <= 1e-3 * np.linalg.norm(yo[sl])
        assert np.linalg.norm(yn64[which][sl] - yno[sl]) <= 1e-10 * np.linalg.norm(yno[sl])
