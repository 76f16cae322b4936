"""Launch settings, the autotuner and multi-mesh groups.  None of them may
change the product: every setting, and a group's single graph launch over
several meshes of uneven size, must give the members' own products bit for
bit."""
import numpy as np
import pytest

import pie_inputs as pi

pytestmark = pytest.mark.gpu

K = 0.01


@pytest.fixture(scope="module")
def pg():
    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    return pg


def columns(n, nrhs, seed):
    import torch
    return torch.from_numpy(np.stack([pi.complex_normal(n, seed + j) for j in range(nrhs)])).cuda()


DEFAULT = dict(overlap=1, near_ctas_per_sm=2, rhs_chunk=1, near_rhs_block=0, far_rows=0, near_kernel=0)
SETTINGS = [dict(DEFAULT, overlap=0, near_ctas_per_sm=0, rhs_chunk=4),
            dict(DEFAULT, near_ctas_per_sm=1, rhs_chunk=4, near_rhs_block=1),
            dict(DEFAULT, near_ctas_per_sm=3, rhs_chunk=2, near_rhs_block=8),
            dict(DEFAULT, near_ctas_per_sm=0, rhs_chunk=1, near_rhs_block=2),
            dict(DEFAULT, overlap=0, near_ctas_per_sm=5, rhs_chunk=3, near_rhs_block=4),
            dict(DEFAULT, rhs_chunk=1, near_kernel=1),
            dict(DEFAULT, overlap=0, rhs_chunk=1, near_kernel=2, far_rows=4)]


@pytest.mark.parametrize("prec", [0, 2])
def test_settings_do_not_change_the_product(pg, prec):
    import torch
    pr = pg.Problem(pg.Mesh(*pi.icosphere(3)), K, 4, root_side=2.0, precision=prec, max_nrhs=4)
    assert pr.tuning == dict(DEFAULT, rhs_chunk=4)
    X = columns(pr.N, 5, 11)
    ref = pr.apply(X)
    torch.cuda.synchronize()
    for s in SETTINGS:
        pr.tuning = s
        assert pr.tuning == s
        assert torch.equal(pr.apply(X), ref), s


def test_tuning_rejects_out_of_range(pg):
    pr = pg.Problem(pg.Mesh(*pi.icosphere(2)), K, 3, root_side=2.0, max_nrhs=2)
    for bad in (dict(overlap=2), dict(near_ctas_per_sm=-1), dict(near_ctas_per_sm=33), dict(rhs_chunk=0),
                dict(rhs_chunk=3), dict(near_rhs_block=3), dict(near_rhs_block=16), dict(far_rows=3),
                dict(far_rows=64), dict(far_rows=-1), dict(near_kernel=3), dict(near_kernel=-1)):
        with pytest.raises(pg.PieError) as ei:
            pr.tuning = bad
        assert ei.value.code == 1
    assert pr.tuning == dict(DEFAULT, rhs_chunk=2)


@pytest.mark.parametrize("prec", [1, 3])
def test_tile_settings_do_not_change_the_small_grid_product(pg, prec):
    """At the inner operator's point (tau = 3, kappa a = 0.15, N_theta = 4,
    P = 32) the far part runs the per-box kernels whose tile far_rows sets,
    and a float near part the kernel near_kernel picks (with 1 to 8
    right-hand sides per pass over the moments): every combination gives
    the default product bit for bit, for one column and for a batch."""
    import torch
    pr = pg.Problem(pg.Mesh(*pi.icosphere(3)), K, 4, root_side=2.0, precision=prec, max_nrhs=4,
                    tau=3, kappa_a=0.15, ntheta=4)
    X = columns(pr.N, 3, 31).to(torch.complex64)
    ref1 = pr.apply(X[0].contiguous())
    ref3 = pr.apply(X)
    torch.cuda.synchronize()
    for rows in (1, 2, 4, 8, 16, 32):
        for nk in (0, 1, 2):
            for ov in (0, 1):
                s = dict(DEFAULT, overlap=ov, rhs_chunk=1, far_rows=rows, near_kernel=nk)
                pr.tuning = s
                assert torch.equal(pr.apply(X[0].contiguous()), ref1), s
        pr.tuning = dict(DEFAULT, rhs_chunk=4, far_rows=rows)
        assert torch.equal(pr.apply(X), ref3), rows
    # several columns per pass: box-staged (1, 2 or 4 columns per block) or
    # warp-per-triangle (1, 2, 4 or 8 per thread)
    for nk in (0, 1, 2):
        for rb in (0, 1, 2, 4, 8):
            s = dict(DEFAULT, rhs_chunk=4, near_rhs_block=rb, near_kernel=nk)
            pr.tuning = s
            assert torch.equal(pr.apply(X), ref3), s



@pytest.mark.parametrize("prec", [1, 2, 3])
def test_near_kernels_agree_on_rows_longer_than_the_staging_buffer(pg, prec):
    """A coarse tree (5120 triangles at L = 3, leaf boxes of 0.25 m: rows of
    more than 512 source triangles) sends the box-staged near kernel down
    its unstaged path, which reads the coefficients of every right-hand side
    from global memory: 1, 2 and 4 columns per block must still give the
    warp-per-triangle kernel's product bit for bit."""
    import torch
    pr = pg.Problem(pg.Mesh(*pi.icosphere(4)), K, 3, root_side=2.0, precision=prec, max_nrhs=4)
    assert pr.near_pairs / pr.T > 512
    dt = torch.complex64 if prec in (1, 3) else torch.complex128
    X = columns(pr.N, 4, 41).to(dt)
    pr.tuning = dict(DEFAULT, rhs_chunk=4, near_rhs_block=4, near_kernel=1)
    ref = pr.apply(X)
    for nk in (0, 2):
        for rb in (1, 2, 4):
            s = dict(DEFAULT, rhs_chunk=4, near_rhs_block=rb, near_kernel=nk)
            pr.tuning = s
            assert torch.equal(pr.apply(X), ref), s
    pr.tuning = dict(DEFAULT, rhs_chunk=1, near_kernel=2)
    assert torch.equal(pr.apply(X), ref)

def test_autotune_keeps_the_product(pg):
    import torch
    pr = pg.Problem(pg.Mesh(*pi.icosphere(3)), K, 4, root_side=2.0, precision=pg.PIE_MIXED, max_nrhs=4)
    X = columns(pr.N, 4, 21)
    ref = pr.apply(X)
    best, ms = pr.autotune(nrhs=4, reps=3)
    assert ms > 0
    assert best == pr.tuning
    assert best["overlap"] in (0, 1) and 0 <= best["near_ctas_per_sm"] <= 32 and 1 <= best["rhs_chunk"] <= 4
    assert best["near_rhs_block"] in (0, 1, 2, 4, 8)
    assert best["far_rows"] in (0, 1, 2, 4, 8, 16, 32) and best["near_kernel"] in (0, 1, 2)
    assert torch.equal(pr.apply(X), ref)


def test_tune_levels_picks_an_admissible_level(pg):
    import torch
    mesh = pg.Mesh(*pi.icosphere(3))
    L, ms = pg.tune_levels(mesh, K, 3, 8, nrhs=1, root_side=2.0, precision=pg.PIE_MIXED)
    # leaf side 2 / 2^(L-1) must stay >= 1.5 x the longest edge (0.165 m here)
    assert set(ms) == {3, 4} and L in ms and ms[L] == min(ms.values())
    x = torch.from_numpy(pi.complex_normal(mesh.nt + mesh.ne, 31)).cuda()
    y3 = pg.Problem(mesh, K, 3, root_side=2.0, precision=pg.PIE_MIXED).apply(x)
    yL = pg.Problem(mesh, K, L, root_side=2.0, precision=pg.PIE_MIXED).apply(x)
    assert (torch.linalg.norm(yL - y3) / torch.linalg.norm(y3)).item() < 1e-3


def group_members(pg):
    return [
        pg.Problem(pg.Mesh(*pi.icosphere(3)), K, 4, root_side=2.0, precision=pg.PIE_FP64, max_nrhs=2),
        pg.Problem(pg.Mesh(*pi.cube(8)), K, 3, root_side=1.0, precision=pg.PIE_MIXED, max_nrhs=3),
        pg.Problem(pg.Mesh(*pi.octasphere(3, (1.0, 0.5, 0.5))), K, 3, precision=pg.PIE_MIXED, max_nrhs=1),
        pg.Problem(pg.Mesh(*pi.cylinder(nseg=16, nrings=2, nrows=8)), K, 3, precision=pg.PIE_FP64, max_nrhs=3),
    ]


def test_group_launch_equals_member_products(pg):
    import torch
    mem = group_members(pg)
    assert len({p.N for p in mem}) == 4
    grp = pg.Group(mem)
    nrhs = 3
    xs = [columns(p.N, nrhs, 40 + 5 * i) for i, p in enumerate(mem)]
    ys = [torch.empty_like(x) for x in xs]
    refs = [p.apply(x) for p, x in zip(mem, xs)]
    grp.apply(xs, ys)
    torch.cuda.synchronize()
    for y, r in zip(ys, refs):
        assert torch.equal(y, r)
    # the same buffers relaunch the captured graph
    for y in ys:
        y.zero_()
    grp.apply(xs, ys)
    torch.cuda.synchronize()
    assert all(torch.equal(y, r) for y, r in zip(ys, refs))
    assert grp.info() == dict(graphs=1, launches=2)
    # a changed member setting is captured anew, with the same result
    mem[0].tuning = dict(overlap=0)
    grp.apply(xs, ys)
    torch.cuda.synchronize()
    assert all(torch.equal(y, r) for y, r in zip(ys, refs))
    assert grp.info() == dict(graphs=2, launches=3)
    # new inputs through the same buffers: the graph reads them
    for x in xs:
        x.mul_(-1j)
    grp.apply(xs, ys)
    torch.cuda.synchronize()
    for y, r in zip(ys, refs):
        # the MIXED members round the near part in float: agree to ~1e-7
        assert (torch.linalg.norm(y + 1j * r) / torch.linalg.norm(r)).item() < 1e-6


def test_group_rejects_bad_arguments(pg):
    mem = group_members(pg)[:2]
    with pytest.raises(pg.PieError):
        pg.Group([mem[0], mem[0]])
    grp = pg.Group(mem)
    mem[1].profile_begin(1)
    import torch
    xs = [columns(p.N, 1, 60 + i) for i, p in enumerate(mem)]
    ys = [torch.empty_like(x) for x in xs]
    with pytest.raises(pg.PieError) as ei:
        grp.apply(xs, ys)
    assert ei.value.code == 1
    mem[1].profile_end()


def test_group_products_match_dense_oracle(pg):
    """Section 8(f2)'s multi-mesh launch against the oracle itself, not only
    against the members' own products: three meshes of uneven size (sphere,
    cube with its faces on box planes, 2:1:1 ellipsoid; 320 / 1536 / 512
    triangles), two right-hand sides each (RWG sources alone, pulse sources
    alone), one graph launch; every member's every column within 1e-3 of the
    oracle's dense Galerkin product per block (the accuracy of Eqs. (4)-(5)
    at the default parameters)."""
    import torch
    from oracle.dense import assemble
    from oracle.mesh import build_topology
    meshes = [(pi.icosphere(2), 2.0), (pi.cube(8), 1.0), (pi.octasphere(3, (1.0, 0.5, 0.5)), 0.0)]
    members, dense = [], []
    for (xyz, tri), side in meshes:
        members.append(pg.Problem(pg.Mesh(xyz, tri), K, 3, root_side=side, precision=pg.PIE_MIXED, max_nrhs=2))
        dense.append(assemble(build_topology(xyz, tri), K))
    assert len({m.T for m in members}) == 3
    xs = []
    for i, m in enumerate(members):
        cols = [np.r_[pi.complex_normal(m.E, 40 + i), np.zeros(m.T)], np.r_[np.zeros(m.E), pi.complex_normal(m.T, 50 + i)]]
        xs.append(torch.from_numpy(np.stack(cols)).cuda())
    ys = [torch.empty_like(x) for x in xs]
    grp = pg.Group(members)
    grp.apply(xs, ys)
    torch.cuda.synchronize()
    assert grp.info()["graphs"] == 1
    for m, Z, x, y in zip(members, dense, xs, ys):
        X, Y = x.cpu().numpy(), y.cpu().numpy()
        for j in range(2):
            yd = Z @ X[j]
            for sl in (slice(0, m.E), slice(m.E, None)):
                err = np.linalg.norm(Y[j][sl] - yd[sl]) / np.linalg.norm(yd[sl])
                assert err < 1e-3, (m.T, j, err)
