"""Brute-force numerical integrals used to pin the oracle's closed forms.

No closed forms here: every integral is a high-order Gauss rule.  In-plane
(or nearly in-plane) singular points are handled by splitting the source
triangle at the projected observation point and collapsing a Gauss rule onto
it, which cancels the 1/R singularity by the polar Jacobian.
"""
import numpy as np

from oracle.quadrature import collapsed_gauss


def inner_reference(r, v, k, n=40):
    """(int_s g, int_s (r' - c_s) g) for point r and triangle v [3,3]."""
    v0, v1, v2 = v
    c = (v0 + v1 + v2) / 3.0
    nrm = np.cross(v1 - v0, v2 - v0)
    nrm /= np.linalg.norm(nrm)
    rho = r - np.dot(r - v0, nrm) * nrm
    b, w = collapsed_gauss(n)
    I0 = 0j
    I1 = np.zeros(3, complex)
    for a, bb in ((v0, v1), (v1, v2), (v2, v0)):
        cr = np.cross(a - rho, bb - rho)
        area = 0.5 * np.dot(cr, nrm)          # signed
        if abs(area) < 1e-300:
            continue
        # collapsed rule: barycentric weight 1 is the collapse vertex (x = u -> 1)
        P = b[:, 0, None] * a + b[:, 1, None] * rho + b[:, 2, None] * bb
        R = np.linalg.norm(P - r, axis=1)
        g = np.exp(1j * k * R) / (4 * np.pi * R)
        I0 += area * np.sum(w * g)
        I1 += area * np.sum((w * g)[:, None] * (P - c), axis=0)
    return I0, I1


def pair_reference(vt, vs, k, n_out=24, n_in=40):
    """(m0, mt, ms, mts) by nested Gauss rules."""
    b, w = collapsed_gauss(n_out)
    ct = vt.mean(axis=0)
    area = 0.5 * np.linalg.norm(np.cross(vt[1] - vt[0], vt[2] - vt[0]))
    P = b @ vt
    m0 = 0j
    mt = np.zeros(3, complex)
    ms = np.zeros(3, complex)
    mts = 0j
    for p, wp in zip(P, w * area):
        K0, K1 = inner_reference(p, vs, k, n_in)
        m0 += wp * K0
        mt += wp * K0 * (p - ct)
        ms += wp * K1
        mts += wp * np.dot(p - ct, K1)
    return m0, mt, ms, mts
