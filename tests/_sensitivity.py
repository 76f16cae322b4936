"""Rounding sensitivity of the oracle MLFMA, the yardstick for the FP64 parity
bars of the CUDA product.

The far part of Eqs. (4)-(5) cancels terms up to ~(2 tau + 1)!! / (kappa w)^tau
times its result in the disaggregation sum, so two FP64 evaluations of the
same discretised operator that differ only in the last bits of their inputs
differ far more than 1e-16 in the product.  These helpers measure how much,
on the oracle alone:

* ``node_sensitivity``: the product's change when the Gauss-Legendre nodes
  and weights of the angular grid (which the CUDA library computes with its
  own Newton iteration) are moved by one unit in the last place;
* ``order_sensitivity``: the change of the per-triangle far potentials when
  the disaggregation sum over the angular samples runs in another order.
"""
import copy

import numpy as np

import oracle.mlfma as mlfma


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def _far_potentials(M, x):
    _, st = M.apply(x, stages=True)
    return np.concatenate([np.ravel(p) for p in M.disaggregate(st["G"][M.L])])


def node_sensitivity(xyz, tri, k, L, x, tau=7, kappa_a=0.08, ntheta=8, side=2.0, seeds=(0, 1), far=False):
    """max over seeds of ||y' - y|| / ||y|| with y' from an oracle whose
    angular nodes and weights carry one-ulp relative perturbations; y is the
    product, or with far=True the per-triangle far potentials (U, V, T1, T2
    concatenated).  Returns (sensitivity, oracle, y)."""
    M = mlfma.MLFMA(xyz, tri, k, L, tau=tau, x=kappa_a, ntheta=ntheta, side=side)
    ev = (lambda O: _far_potentials(O, x)) if far else (lambda O: O.apply(x))
    y = ev(M)
    orig = mlfma.angular_grid
    out = 0.0
    for seed in seeds:
        rng = np.random.default_rng(seed)

        def grid(n, rng=rng):
            c, w = np.polynomial.legendre.leggauss(n)
            c = c * (1 + rng.choice([-1.0, 1.0], c.shape) * 2.0 ** -53)
            w = w * (1 + rng.choice([-1.0, 1.0], w.shape) * 2.0 ** -53)
            nphi = 2 * n
            ct = np.repeat(c, nphi)
            st = np.sqrt(1.0 - ct * ct)
            ph = np.tile(np.pi * np.arange(nphi) / n, n)
            return np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1), np.repeat(w, nphi) * (np.pi / n)

        mlfma.angular_grid = grid
        try:
            Mp = mlfma.MLFMA(xyz, tri, k, L, tau=tau, x=kappa_a, ntheta=ntheta, side=side)
        finally:
            mlfma.angular_grid = orig
        out = max(out, _rel(ev(Mp), y))
    return out, M, y


def hankel_sensitivity(xyz, tri, k, L, x, tau=7, kappa_a=0.08, ntheta=8, side=2.0, seeds=(0, 1)):
    """max over seeds of the product's relative change when every scaled
    Hankel value s^t h_t(k|w|) of Eq. (5) carries a one-ulp relative
    perturbation (two valid FP64 evaluations of h_t differ by a few ulps)."""
    import oracle.asd as asd
    M = mlfma.MLFMA(xyz, tri, k, L, tau=tau, x=kappa_a, ntheta=ntheta, side=side)
    y = M.apply(x)
    orig = asd.scaled_hankel
    out = 0.0
    for seed in seeds:
        rng = np.random.default_rng(seed)

        def hankel(t, z, s, rng=rng):
            H = orig(t, z, s)
            return H * (1 + 2.0 ** -53 * (rng.choice([-1.0, 1.0], H.shape) + 1j * rng.choice([-1.0, 1.0], H.shape)))

        asd.scaled_hankel = hankel
        try:
            Mp = mlfma.MLFMA(xyz, tri, k, L, tau=tau, x=kappa_a, ntheta=ntheta, side=side)
        finally:
            asd.scaled_hankel = orig
        out = max(out, _rel(Mp.apply(x), y))
    return out


def order_sensitivity(M, GL, seeds=(0, 1)):
    """max over seeds of the relative change of M.disaggregate(GL) (all four
    potentials together) when the samples are summed in a random order."""
    ref = np.concatenate([np.ravel(p) for p in M.disaggregate(GL)])
    out = 0.0
    for seed in seeds:
        perm = np.random.default_rng(seed).permutation(M.P)
        Mp = copy.copy(M)
        Mp.Pi = M.Pi[:, perm]
        Mp.M = M.M[:, :, perm]
        got = np.concatenate([np.ravel(p) for p in Mp.disaggregate(GL[:, :, perm])])
        out = max(out, _rel(got, ref))
    return out
