"""The open-patch experiment of Section 4 (Fig. 1): a PEC square patch with
0.6 m edges at 1 MHz and 100 MHz, x-polarised plane wave propagating along z,
solved with MLFMA at 3, 4, 5 and 6 levels; the far-zone field on the z-x plane
must agree between level counts within the 0.3 dB window of the figure
(compared where the field is within 40 dB of its maximum).  The mesh is a
uniform 75 x 75 grid of split squares: 11,250 pulses as in the paper, 16,725
RWG functions (a uniform grid cannot give the paper's 16,250)."""
import numpy as np
import pytest

import pie_inputs as pi

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("freq", [1e6, 1e8])
def test_patch_levels_agree(freq):
    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    xyz, tri = pi.square_patch(75)
    k = 2 * np.pi * freq / 299792458.0
    mesh = pg.Mesh(xyz, tri)
    assert mesh.nt == 11250
    rh = pi.bistatic_directions(181)
    fields = {}
    for L in (3, 4, 5, 6):
        pr = pg.Problem(mesh, k, L, precision=pg.PIE_MIXED)
        b = pr.rhs_planewave([0, 0, 1.0], [1.0, 0, 0])
        x, st = pr.solve(b, tol=1e-5, maxit=4000, restart=300)
        assert st["converged"], (L, st)
        E = pr.farfield(x, rh).cpu().numpy()
        fields[L] = 10 * np.log10(np.sum(np.abs(E) ** 2, axis=1))
        print(freq, L, "iterations", st["iterations"])
    ref = fields[6]
    mask = ref > ref.max() - 40
    for L in (3, 4, 5):
        dev = np.max(np.abs(fields[L][mask] - ref[mask]))
        print(freq, L, "max deviation from 6 levels (dB)", dev)
        assert dev < 0.3


def test_patch_standard_diagonalization_matches_oracle():
    """The capped scale factor of the Fig. 1 study at 100 MHz: boxes larger
    than x / k0 in wavelengths use s = 1 (the standard diagonalization of
    Eq. (4)), here at every level of a 200-triangle patch at 3 levels (leaf
    0.15 m, k0 a = 0.31 > 0.08) and an 800-triangle one at 4 levels.  GPU stages against the oracle MLFMA with the same
    scale factors per level and component to 1e-12, the product against it
    within 16 x the oracle's own sensitivity to one-ulp changes of its
    angular nodes or of its scaled Hankel values (about 1e-9 here), and
    against the oracle's dense product to 1e-3 per block."""
    import torch
    from oracle.dense import assemble
    from tests._lib import ensure_built
    from tests._sensitivity import hankel_sensitivity, node_sensitivity
    ensure_built()
    import paper_1806_04164_gb300 as pg
    from oracle.mlfma import MLFMA
    k = 2 * np.pi * 1e8 / 299792458.0
    for n, L in ((10, 3), (20, 4)):
        xyz, tri = pi.square_patch(n)
        M = MLFMA(xyz, tri, k, L)
        assert all(M.scale[l] == 1.0 for l in range(3, L + 1))
        pr = pg.Problem(pg.Mesh(xyz, tri), k, L)
        x = pi.complex_normal(pr.N, 9)
        y = pr.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        yo, st = M.apply(x, stages=True)
        rel = lambda a, b: np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))
        for l in range(3, L + 1):
            # per component against the level's pattern norm (the flat patch
            # radiates no z current: that component is zero on both sides)
            S, G = pr.stage(0, l), pr.stage(1, l)
            nS, nG = np.linalg.norm(st["S"][l]), np.linalg.norm(st["G"][l])
            for c in range(5):
                assert np.linalg.norm(S[:, c] - st["S"][l][:, c]) <= 1e-12 * nS, ("S", L, l, c)
                assert np.linalg.norm(G[:, c] - st["G"][l][:, c]) <= 1e-12 * nG, ("G", L, l, c)
        sens, _, _ = node_sensitivity(xyz, tri, k, L, x, side=0.0)
        hs = hankel_sensitivity(xyz, tri, k, L, x, side=0.0)
        print(f"patch L={L}: GPU vs oracle {rel(y, yo):.2e}, node sensitivity {sens:.2e}, Hankel {hs:.2e}")
        # at s = 1 the translation terms are moderate (k0 |w| up to 1.6), and
        # the GPU's recurrences for h_t and P_t and scipy's routines differ by
        # several ulps: measured 12 x the one-ulp sensitivities at L = 3
        assert rel(y, yo) <= 16 * max(sens, hs)
        Z = assemble(M.top, k)
        for xx in (np.r_[pi.complex_normal(pr.E, 1), np.zeros(pr.T)], np.r_[np.zeros(pr.E), pi.complex_normal(pr.T, 2)]):
            ym = pr.apply(torch.from_numpy(xx).cuda()).cpu().numpy()
            yd = Z @ xx
            for sl in (slice(0, pr.E), slice(pr.E, None)):
                assert rel(ym[sl], yd[sl]) < 1e-3, (L, rel(ym[sl], yd[sl]))
