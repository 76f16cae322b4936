"""Pins for oracle.mie (PEC sphere)."""
import numpy as np

from oracle import mie


def test_rayleigh_limit():
    R = 1.0
    for k in (1e-2, 1e-3):
        g = np.linspace(0, np.pi, 37)
        c = np.cos(g)
        se = mie.rcs_eplane(k, R, c)
        sh = mie.rcs_hplane(k, R, c)
        x4 = (k * R) ** 4
        re = 4 * np.pi * R * R * x4 * (c - 0.5) ** 2
        rh = 4 * np.pi * R * R * x4 * (1 - 0.5 * c) ** 2
        scale = 4 * np.pi * R * R * x4
        assert np.max(np.abs(se - re)) < 10 * (k * R) ** 2 * scale
        assert np.max(np.abs(sh - rh)) < 10 * (k * R) ** 2 * scale
        assert abs(mie.rcs_eplane(k, R, -1.0) / (9 * np.pi * R * R * x4) - 1) < 10 * (k * R) ** 2


def test_optical_theorem_and_angular_integral():
    for x in (0.3, 1.0, 3.0):
        ext, sca = mie.cross_sections(x, 1.0)
        assert abs(ext - sca) < 1e-10 * sca
        mu, wmu = np.polynomial.legendre.leggauss(200)
        S1, S2 = mie.amplitudes(x, mu)
        # unpolarised average over azimuth: (|S1|^2 + |S2|^2)/2, times 2 pi, / k^2
        tot = np.pi * np.sum(wmu * (np.abs(S1) ** 2 + np.abs(S2) ** 2)) / x ** 2
        assert abs(tot - sca) < 1e-8 * sca
