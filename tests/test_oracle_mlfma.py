"""Pins for oracle.mlfma (the MVM of Section 3)."""
import numpy as np
import pytest
from scipy.special import eval_legendre

import pie_inputs as pi
from oracle.asd import angular_grid
from oracle.dense import assemble
from oracle.mesh import build_topology
from oracle.mlfma import MLFMA, interpolation_filter


@pytest.fixture(scope="module")
def case():
    xyz, tri = pi.icosphere(2)
    k = 0.01
    M = MLFMA(xyz, tri, k, 3, side=2.0)
    top = M.top
    Z = assemble(top, k)
    tr = M.tree
    leaf = np.empty(top.T, np.int64)
    leaf[tr.perm] = np.repeat(np.arange(tr.keys[3].size), np.diff(tr.leaf_start))
    ijk = tr.ijk[3][leaf]

    def near(t, s):
        return np.max(np.abs(ijk[t] - ijk[s]), axis=1) <= 1

    Zn = assemble(top, k, pair_mask=near)
    return M, Z, Zn


def test_near_part_is_exact(case):
    M, Z, Zn = case
    x = pi.complex_normal(M.top.N, 21)
    y = M.apply(x, far=False)
    assert np.linalg.norm(y - Zn @ x) <= 1e-12 * np.linalg.norm(Zn @ x)


def test_far_part_within_asd_accuracy(case):
    M, Z, Zn = case
    E = M.top.E
    for x in (np.r_[pi.complex_normal(E, 1), np.zeros(M.top.T)], np.r_[np.zeros(E), pi.complex_normal(M.top.T, 2)]):
        yd = Z @ x
        ym = M.apply(x)
        for sl in (slice(0, E), slice(E, None)):
            assert np.linalg.norm(ym[sl] - yd[sl]) <= 1e-3 * np.linalg.norm(yd[sl])
        # and the far field is a large part of the product
        yn = M.apply(x, far=False)
        assert np.linalg.norm(yd - yn) > 0.1 * np.linalg.norm(yd)


def test_filter_against_legendre_addition_theorem():
    nt = 5
    khat, w = angular_grid(nt)
    F = interpolation_filter(khat, w, nt, 0.5)
    cosang = np.clip(khat @ khat.T, -1, 1)
    ref = np.zeros_like(F)
    for l in range(nt):
        ref += 0.5 ** l * (2 * l + 1) / (4 * np.pi) * eval_legendre(l, cosang) * w[None, :]
    assert np.allclose(F, ref, atol=1e-13)
    # ratio 1 is the projector onto degree < nt: idempotent
    P1 = interpolation_filter(khat, w, nt, 1.0)
    assert np.allclose(P1 @ P1, P1, atol=1e-12)


def test_multilevel_far_part():
    """Four levels (interpolation and anterpolation in use) on the
    1280-triangle sphere, checked on sampled outputs computed row by row."""
    from oracle.dense import rows
    xyz, tri = pi.icosphere(3)
    M = MLFMA(xyz, tri, 0.01, 4, side=2.0)
    x = pi.complex_normal(M.top.N, 4)
    x[M.top.E:] *= 1e-3
    which = np.random.default_rng(9).choice(M.top.N, 60, replace=False)
    yd = rows(M.top, 0.01, which, x)
    ym = M.apply(x)[which]
    assert np.linalg.norm(ym - yd) <= 1e-3 * np.linalg.norm(yd)


def test_rejects_leaf_smaller_than_near_singular_radius():
    xyz, tri = pi.icosphere(2)
    with pytest.raises(ValueError):
        MLFMA(xyz, tri, 0.01, 4, side=2.0)


def test_far_part_reciprocity():
    """The discrete far part is complex symmetric in exact arithmetic: with
    low-amplification parameters u^T M v = v^T M u to ~1e-13 (at the chosen
    parameters the FP64 rounding amplification leaves ~1e-5)."""
    xyz, tri = pi.icosphere(3)
    M = MLFMA(xyz, tri, 0.01, 4, tau=3, x=0.4, ntheta=4, side=2.0)
    u = pi.complex_normal(M.top.N, 1)
    v = pi.complex_normal(M.top.N, 2)
    a = u @ M.apply(v, near=False)
    b = v @ M.apply(u, near=False)
    assert abs(a - b) <= 1e-12 * abs(a)
    an = u @ M.apply(v, far=False)
    bn = v @ M.apply(u, far=False)
    assert abs(an - bn) <= 1e-13 * abs(an)


@pytest.mark.parametrize("freq", [1e6, 1e8])
def test_open_patch_both_regimes(freq):
    """Open surface (boundary edges carry no RWG) at 1 MHz (scaled plane waves,
    s = 0.04) and 100 MHz (leaf boxes at s = 1, the standard diagonalization):
    far part within 1e-3 of the dense product per block."""
    xyz, tri = pi.square_patch(10)
    k = 2 * np.pi * freq / 299792458.0
    M = MLFMA(xyz, tri, k, 3)
    Z = assemble(M.top, k)
    E = M.top.E
    for x in (np.r_[pi.complex_normal(E, 1), np.zeros(M.top.T)], np.r_[np.zeros(E), pi.complex_normal(M.top.T, 2)]):
        yd, ym = Z @ x, M.apply(x)
        for sl in (slice(0, E), slice(E, None)):
            assert np.linalg.norm(ym[sl] - yd[sl]) <= 1e-3 * np.linalg.norm(yd[sl])
