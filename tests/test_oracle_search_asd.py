"""Pins for oracle.search_asd: the Eq. (4)-(5) error in FP64 and in emulated
FP32, and the rounding amplification that decides which arithmetic a
parameter point tolerates."""
import numpy as np

from oracle.search_asd import (EPS32, EPS64, amplification, eq4_terms, exact_g, geometries, green_fp32,
                               green_fp64, pair_errors)

K, A = 1e-3, 0.0625   # a leaf box of the 81,920-triangle sphere at kR = 1e-3 (k a = 6.25e-5)


def test_fp32_equals_fp64_without_amplification():
    """tau = 2: the Eq. (5) terms stay within a few hundred times g, so
    float rounding stays at ~1e-5 and both arithmetics show the same error
    (the truncation error of tau = 2)."""
    r64, m64 = pair_errors(K, A, 0.2, 2, 4, npair=20, npts=15)
    r32, m32 = pair_errors(K, A, 0.2, 2, 4, npair=20, npts=15, fp32=True)
    assert abs(r32 - r64) < 1e-5 and abs(m32 - m64) < 1e-4


def test_fp32_excess_bounded_by_amplification():
    """Per point pair, |g_32 - g_64| / |g| <= 8 eps_32 cond (the rounding of
    each summand, of its phase factors and of the running sum is a few eps
    of that summand), and at the FP64 point (tau 7, x 0.08) the excess is
    large: the cancellation is real, not an artefact of the estimate."""
    for tau, nth, x in ((4, 6, 0.1), (7, 8, 0.08), (7, 8, 0.2)):
        s = K * A / x
        for Co, Cs, r, rp in geometries(A, 6, 10, seed=3):
            g = exact_g(K, r, rp)
            d = np.abs(green_fp32(K, s, tau, nth, r, rp, Co, Cs) - green_fp64(K, s, tau, nth, r, rp, Co, Cs))
            al, po, ps = eq4_terms(K, s, tau, nth, r, rp, Co, Cs)
            cond_pair = (np.abs(po * ps) @ np.abs(al)) / np.abs(g)
            assert np.all(d / np.abs(g) <= 8 * EPS32 * cond_pair)
    r32, _ = pair_errors(K, A, 0.08, 7, 8, npair=10, npts=10, fp32=True)
    assert r32 > 1.0     # FP32 at the FP64 point: no correct digit


def test_scaled_wave_error_grows_as_x_squared():
    """At low frequency the Eq. (4) error (tau large enough that truncation
    is negligible) is the first neglected term of s^t j_t(z/s) ~ j_t(z),
    relative size (kappa v)^2 / (2 (2t + 3)): doubling x = kappa a multiplies
    it by 4."""
    e = {x: pair_errors(K, A, x, 7, 10, npair=30, npts=15)[0] for x in (0.1, 0.2, 0.15, 0.3)}
    assert 3.5 < e[0.2] / e[0.1] < 4.5
    assert 3.5 < e[0.3] / e[0.15] < 4.5


def test_amplification_matches_leading_hankel_term():
    """cond grows like (2 tau + 1)!! / (kappa w)^tau: at fixed tau, halving x
    multiplies it by about 2^tau."""
    c1 = amplification(K, A, 0.2, 5, 6, npair=20, npts=10)
    c2 = amplification(K, A, 0.1, 5, 6, npair=20, npts=10)
    assert 0.7 * 2 ** 5 < c2 / c1 < 1.3 * 2 ** 5


def test_chosen_points():
    """The library's FP64 point (tau 7, x 0.08, N_theta 8) keeps the Eq. (4)
    error below 1e-3 RMS with its FP64 rounding term eps_64 cond below 1e-4;
    the FP32 point of the nested solver's inner operator (tau 4, x 0.1,
    N_theta 6) keeps the emulated-FP32 error below 3e-3 RMS and 3e-2 max."""
    r64, m64 = pair_errors(K, A, 0.08, 7, 8, npair=40, npts=20)
    assert r64 < 1e-3 and m64 < 5e-3
    assert EPS64 * amplification(K, A, 0.08, 7, 8, npair=40, npts=20) < 1e-4
    r32, m32 = pair_errors(K, A, 0.1, 4, 6, npair=40, npts=20, fp32=True)
    assert r32 < 3e-3 and m32 < 3e-2
    # same error at another box size in wavelengths (stable as k a -> 0)
    r32b, _ = pair_errors(1e-2, 0.5, 0.1, 4, 6, npair=40, npts=20, fp32=True)
    assert abs(r32b - r32) < 0.2 * r32
