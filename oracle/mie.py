"""Mie series for a perfectly conducting sphere (Section 4 compares the sphere
solutions with "analytical results obtained via a Mie-series solution").

Written from the textbook series (Bohren & Huffman 1983, ch. 4, with the
perfect-conductor limit of the coefficients), exp(-i w t):
  a_n = [x j_n(x)]' / [x h_n(x)]',  b_n = j_n(x) / h_n(x),  x = k R, h_n = j_n + i y_n
  S1 = sum (2n+1)/(n(n+1)) (a_n pi_n + b_n tau_n),  S2 = sum (2n+1)/(n(n+1)) (a_n tau_n + b_n pi_n)
with pi_n, tau_n from the usual upward recurrences in mu = cos(gamma).
Bistatic RCS: sigma_E = 4 pi |S2|^2 / k^2 in the E-plane, sigma_H = 4 pi |S1|^2 / k^2
in the H-plane.  Spherical Bessel functions are scipy.special routines.

Pinned in tests/test_oracle_mie.py: the Rayleigh limit
(sigma_E = 4 pi R^2 (kR)^4 (cos g - 1/2)^2, sigma_H = 4 pi R^2 (kR)^4 (1 - cos g / 2)^2),
the optical theorem (extinction = scattering for a lossless sphere), and the
angular integral of |S1|^2 + |S2|^2 against the total scattering cross-section.
"""
import numpy as np
from scipy.special import spherical_jn, spherical_yn


def nmax_of(x):
    return max(3, int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 2.0)))


def coefficients(x, nmax=None):
    nmax = nmax or nmax_of(x)
    n = np.arange(1, nmax + 1)
    j = spherical_jn(n, x)
    jp = spherical_jn(n, x, derivative=True)
    y = spherical_yn(n, x)
    yp = spherical_yn(n, x, derivative=True)
    h = j + 1j * y
    hp = jp + 1j * yp
    a = (j + x * jp) / (h + x * hp)
    b = j / h
    return n, a, b


def amplitudes(x, cosg, nmax=None):
    n, a, b = coefficients(x, nmax)
    mu = np.asarray(cosg, np.float64)
    pi_prev = np.zeros_like(mu)
    pi_cur = np.ones_like(mu)
    S1 = np.zeros(mu.shape, np.complex128)
    S2 = np.zeros(mu.shape, np.complex128)
    for i, nn in enumerate(n):
        tau = nn * mu * pi_cur - (nn + 1) * pi_prev
        f = (2 * nn + 1) / (nn * (nn + 1))
        S1 += f * (a[i] * pi_cur + b[i] * tau)
        S2 += f * (a[i] * tau + b[i] * pi_cur)
        pi_next = ((2 * nn + 1) * mu * pi_cur - (nn + 1) * pi_prev) / nn
        pi_prev, pi_cur = pi_cur, pi_next
    return S1, S2


def rcs_eplane(k, R, cosg):
    _, S2 = amplitudes(k * R, cosg)
    return 4.0 * np.pi * np.abs(S2) ** 2 / k ** 2


def rcs_hplane(k, R, cosg):
    S1, _ = amplitudes(k * R, cosg)
    return 4.0 * np.pi * np.abs(S1) ** 2 / k ** 2


def cross_sections(k, R):
    """(extinction, scattering) cross-sections."""
    n, a, b = coefficients(k * R)
    ext = 2 * np.pi / k ** 2 * np.sum((2 * n + 1) * np.real(a + b))
    sca = 2 * np.pi / k ** 2 * np.sum((2 * n + 1) * (np.abs(a) ** 2 + np.abs(b) ** 2))
    return ext, sca
