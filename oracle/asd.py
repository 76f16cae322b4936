"""Approximate stable diagonalization of the Green's function, Eqs. (4)-(5).

Eq. (4): with r - r' = w + v and a scale factor s,
    g(r, r') ~ (i k / (16 pi^2)) sum_p w_p exp(i (k/s) khat_p . v) alpha(k, khat_p, w)
Eq. (5):
    alpha(k, khat, w) = sum_{t=0}^{tau} i^t (2t+1) s^t h_t^(1)(k|w|) P_t(khat . what).

Reading of the prefactor (the paper prints i k0 / (4 pi) in front of an angular
integral): with the unnormalised solid-angle measure (sum_p w_p = 4 pi) the
plane-wave expansion and Gegenbauer's addition theorem give i k / (16 pi^2);
i k / (4 pi) is the same with the integral read as a mean over the sphere.
Pinned: with s = 1 and large tau the formula reproduces g to ~1e-12 for
well-separated points (tests/test_oracle_asd.py).

Angular samples (reading): N_theta Gauss-Legendre nodes in cos(theta)
(ascending) times 2 N_theta uniform azimuths phi_j = pi j / N_theta; sample
index p = i_theta * 2 N_theta + j_phi; weights w_theta * pi / N_theta.  This
rule integrates spherical harmonics exactly up to degree 2 N_theta - 1.

Spherical Bessel functions and Legendre polynomials come from scipy.special.
"""
import numpy as np
from scipy.special import eval_legendre, spherical_jn, spherical_yn


def angular_grid(ntheta: int):
    x, wx = np.polynomial.legendre.leggauss(ntheta)
    nphi = 2 * ntheta
    phi = np.pi * np.arange(nphi) / ntheta
    ct = np.repeat(x, nphi)
    st = np.sqrt(1.0 - ct * ct)
    ph = np.tile(phi, ntheta)
    khat = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    w = np.repeat(wx, nphi) * (np.pi / ntheta)
    return khat, w


def scaled_hankel(tau: int, z, s):
    """s^t h_t^(1)(z) for t = 0..tau (complex, shape [tau+1] + z.shape)."""
    z = np.asarray(z, np.float64)
    out = []
    for t in range(tau + 1):
        out.append((s ** t) * (spherical_jn(t, z) + 1j * spherical_yn(t, z)))
    return np.array(out)


def alpha_tilde(k, s, tau, wvec, khat):
    """Eq. (5) for one separation vector wvec [3] at directions khat [P,3]."""
    wvec = np.asarray(wvec, np.float64)
    wn = np.linalg.norm(wvec)
    cosang = khat @ (wvec / wn)
    H = scaled_hankel(tau, k * wn, s)
    out = np.zeros(khat.shape[0], np.complex128)
    for t in range(tau + 1):
        out += (1j ** t) * (2 * t + 1) * H[t] * eval_legendre(t, cosang)
    return out


def green_asd(k, s, tau, ntheta, r, rp, Co, Cs):
    """Eq. (4) evaluated for point pairs r [M,3], rp [M,3] in boxes centred at
    Co (observation) and Cs (source), one box pair (Co, Cs fixed)."""
    khat, w = angular_grid(ntheta)
    wvec = np.asarray(Co, float) - np.asarray(Cs, float)
    alpha = alpha_tilde(k, s, tau, wvec, khat)
    v = (np.asarray(r) - Co) - (np.asarray(rp) - Cs)            # [M,3]
    ph = np.exp(1j * (k / s) * (v @ khat.T))                     # [M,P]
    return (1j * k / (16.0 * np.pi ** 2)) * (ph @ (w * alpha))


def far_offsets():
    """The 316 box-index offsets of a one-box-buffer interaction list:
    {-3..3}^3 without {-1..1}^3, ordered by (dx, dy, dz) lexicographically."""
    out = []
    for dx in range(-3, 4):
        for dy in range(-3, 4):
            for dz in range(-3, 4):
                if max(abs(dx), abs(dy), abs(dz)) > 1:
                    out.append((dx, dy, dz))
    return np.array(out, dtype=np.int64)
