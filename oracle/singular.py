"""Analytic potential integrals over a planar triangle (near-singular entries).

After the integration by parts of Section 3 the only kernel of the PIEs is
g = exp(i k0 R) / (4 pi R) (Section 2).  For triangle pairs that touch or lie
close together the inner integral is split as g = 1/(4 pi R) + (exp(ikR)-1)/(4 pi R):
the first part is integrated in closed form, the second (smooth) part by
quadrature.  The closed forms are the classical ones for a flat triangle
(Wilton et al., IEEE TAP 1984; Graglia, IEEE TAP 1993), written here from the
geometry: with unit normal n, signed height d = n.(r - v0), and for every edge
(a -> b, counter-clockwise) its unit tangent s, outward in-plane normal
m = s x n, l+ = (b - r).s, l- = (a - r).s, P0 = (a - r).m, R+- = |r - b|, |r - a|,
R0^2 = P0^2 + d^2 and f = ln((R+ + l+)/(R- + l-)):

  int 1/R dS'          = sum_e [ P0 f - |d| (atan(P0 l+/(R0^2+|d|R+)) - atan(P0 l-/(R0^2+|d|R-))) ]
  int (rho'-rho)/R dS' = 1/2 sum_e m [ R0^2 f + l+ R+ - l- R- ]
  int (r'-r)/R dS'     = int (rho'-rho)/R dS' - d n int 1/R dS'.

Pinned in tests/test_oracle_singular.py against high-order numerical
integration (off-plane points: plain Gauss; in-plane points: the triangle split
at the observation point, each piece in polar Duffy coordinates).
"""
import numpy as np


def _log_ratio(Rp, lp, Rm, lm, R02, elen):
    """ln((R+ + l+)/(R- + l-)) in a cancellation-free form; 0 where R0 is zero
    to rounding (the point lies on the edge's line, where the factors P0 and
    R0^2 that multiply this logarithm vanish)."""
    out = np.zeros(np.broadcast(Rp, lp, Rm, lm, R02, elen).shape)
    Rp, lp, Rm, lm, R02, elen = np.broadcast_arrays(Rp, lp, Rm, lm, R02, elen)
    tiny = R02 <= 1e-24 * elen * elen
    c1 = (lm >= 0) & ~tiny
    c2 = (lp <= 0) & ~tiny & ~c1
    c3 = ~(c1 | c2 | tiny)
    out[c1] = np.log((Rp[c1] + lp[c1]) / (Rm[c1] + lm[c1]))
    out[c2] = np.log((Rm[c2] - lm[c2]) / (Rp[c2] - lp[c2]))
    out[c3] = np.log((Rp[c3] + lp[c3]) * (Rm[c3] - lm[c3]) / R02[c3])
    return out


def potential_integrals(r, v0, v1, v2):
    """Closed-form I1 = int_T 1/|r-r'| dS' and Ir = int_T (r'-r)/|r-r'| dS'.

    r, v0, v1, v2 broadcast over leading axes ([...,3]).  Returns (I1 [...],
    Ir [...,3]).
    """
    r = np.asarray(r, np.float64)
    v0, v1, v2 = (np.asarray(v, np.float64) for v in (v0, v1, v2))
    cr = np.cross(v1 - v0, v2 - v0)
    n = cr / np.linalg.norm(cr, axis=-1, keepdims=True)
    d = np.sum(n * (r - v0), axis=-1)
    ad = np.abs(d)
    I1 = np.zeros(np.broadcast(d, r[..., 0]).shape)
    Ip = np.zeros(I1.shape + (3,))
    for a, b in ((v0, v1), (v1, v2), (v2, v0)):
        e = b - a
        elen = np.linalg.norm(e, axis=-1)
        s = e / elen[..., None]
        m = np.cross(s, n)
        lp = np.sum((b - r) * s, axis=-1)
        lm = np.sum((a - r) * s, axis=-1)
        P0 = np.sum((a - r) * m, axis=-1)
        Rp = np.linalg.norm(r - b, axis=-1)
        Rm = np.linalg.norm(r - a, axis=-1)
        R02 = P0 * P0 + d * d
        f = _log_ratio(Rp, lp, Rm, lm, R02, elen)
        den_p = R02 + ad * Rp
        den_m = R02 + ad * Rm
        with np.errstate(divide="ignore", invalid="ignore"):
            at = np.where(den_p > 0, np.arctan(P0 * lp / np.where(den_p > 0, den_p, 1.0)), 0.0) \
                - np.where(den_m > 0, np.arctan(P0 * lm / np.where(den_m > 0, den_m, 1.0)), 0.0)
        I1 = I1 + P0 * f - ad * at
        Ip = Ip + 0.5 * m * (R02 * f + lp * Rp - lm * Rm)[..., None]
    Ir = Ip - (d * I1)[..., None] * n
    return I1, Ir
