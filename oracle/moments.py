"""Per-triangle-pair moments of the Green's function (Sections 2-3).

After the integration by parts of Section 3 every Galerkin entry of Eqs. (1)-(2)
is a combination of four double integrals over a test triangle t and a source
triangle s, with local coordinates u = r - c_t and u' = r' - c_s (c = centroid):

  m0  = int_t int_s g            mt  = int_t int_s u g   (3-vector)
  ms  = int_t int_s u' g (3-vec) mts = int_t int_s u.u' g

with g = exp(i k0 R) / (4 pi R), R = |r - r'| (Section 2).

Rules (readings; the paper does not state its integration rules):
* regular pairs: the 7-point degree-5 rule on both triangles;
* near-singular pairs, defined by |c_t - c_s|^2 < 2.25 max(h_t^2, h_s^2) with h
  the longest edge of a triangle: outer 64-point (8 x 8) collapsed Gauss rule on t; the
  inner integral over s split as 1/(4 pi R) (closed form, oracle.singular) plus
  (exp(i k R) - 1)/(4 pi R) by the 7-point rule; the rule is applied in both
  orders and averaged (m0, mts symmetric; mt(t,s) with ms(s,t)), so that the
  discrete operator keeps the reciprocity Z^T = Z of the continuous Galerkin
  operator (the one-sided rule breaks it at ~1e-4).
The squared distances and edge lengths are formed as ((x*x + y*y) + z*z) in
IEEE double without fused multiply-add, so the classification is reproducible.

Pinned in tests/test_oracle_moments.py (near-singular rule against brute-force
nested adaptive integration on two-triangle meshes; symmetry of m0 and mts and
the swap mt(t,s) = ms(s,t); the k -> 0 limit against the static 1/(4 pi R)).
"""
import numpy as np

from .quadrature import collapsed_gauss, radon7
from .singular import potential_integrals

FOUR_PI = 4.0 * np.pi


def sq3(d):
    """((x*x + y*y) + z*z) along the last axis, no contraction."""
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def max_edge2(xyz, tri):
    v0, v1, v2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    return np.maximum(np.maximum(sq3(v1 - v0), sq3(v2 - v1)), sq3(v0 - v2))


def is_near_singular(cent, h2, t, s):
    """Pair classification used by the dense operator (see module header)."""
    d2 = sq3(cent[t] - cent[s])
    return d2 < 2.25 * np.maximum(h2[t], h2[s])


def green_remainder(k, R):
    """(exp(i k R) - 1) / (4 pi R), evaluated without cancellation."""
    R = np.asarray(R, np.float64)
    safe = np.where(R > 0, R, 1.0)
    kr = k * safe
    sh = np.sin(0.5 * kr)
    val = (-2.0 * sh * sh + 1j * np.sin(kr)) / (FOUR_PI * safe)
    return np.where(R > 0, val, 1j * k / FOUR_PI)


def green(k, R):
    return np.exp(1j * k * R) / (FOUR_PI * R)


class Geometry:
    """Per-triangle data shared by the moment rules."""

    def __init__(self, xyz, tri):
        self.xyz = np.asarray(xyz, np.float64)
        self.tri = np.asarray(tri, np.int64)
        v0, v1, v2 = (self.xyz[self.tri[:, i]] for i in range(3))
        self.v = np.stack([v0, v1, v2], axis=1)           # [T,3,3]
        self.area = 0.5 * np.linalg.norm(np.cross(v1 - v0, v2 - v0), axis=1)
        self.cent = (v0 + v1 + v2) / 3.0
        self.h2 = max_edge2(self.xyz, self.tri)
        b7, w7 = radon7()
        self.q7 = np.einsum("qk,tkd->tqd", b7, self.v)    # [T,7,3]
        self.w7 = w7[None, :] * self.area[:, None]         # [T,7]
        b64, w64 = collapsed_gauss(8)
        self.q64 = np.einsum("qk,tkd->tqd", b64, self.v)  # [T,64,3]
        self.w64 = w64[None, :] * self.area[:, None]


def regular_moments(geo: Geometry, k, t, s):
    """Moments by the 7 x 7 product rule for pair arrays t, s."""
    rt, wt = geo.q7[t], geo.w7[t]                 # [P,7,3], [P,7]
    rs, ws = geo.q7[s], geo.w7[s]
    ut = rt - geo.cent[t][:, None, :]
    us = rs - geo.cent[s][:, None, :]
    R = np.linalg.norm(rt[:, :, None, :] - rs[:, None, :, :], axis=-1)  # [P,7,7]
    G = green(k, R) * wt[:, :, None] * ws[:, None, :]
    m0 = G.sum(axis=(1, 2))
    mt = np.einsum("pij,pid->pd", G, ut)
    ms = np.einsum("pij,pjd->pd", G, us)
    mts = np.einsum("pij,pid,pjd->p", G, ut, us)
    return m0, mt, ms, mts


def singular_moments(geo: Geometry, k, t, s):
    """Moments with the closed-form static inner integral (near pairs)."""
    ri, Wi = geo.q64[t], geo.w64[t]               # [P,64,3], [P,64]
    vs = geo.v[s]                                  # [P,3,3]
    cs = geo.cent[s][:, None, :]
    I1, Ir = potential_integrals(ri, vs[:, None, 0], vs[:, None, 1], vs[:, None, 2])
    rj, wj = geo.q7[s], geo.w7[s]                 # [P,7,3]
    R = np.linalg.norm(ri[:, :, None, :] - rj[:, None, :, :], axis=-1)  # [P,64,7]
    rem = green_remainder(k, R) * wj[:, None, :]
    K0 = I1 / FOUR_PI + rem.sum(axis=2)
    K1 = (Ir + (ri - cs) * I1[..., None]) / FOUR_PI + np.einsum("pij,pjd->pid", rem, rj - cs)
    ut = ri - geo.cent[t][:, None, :]
    m0 = np.einsum("pi,pi->p", Wi, K0)
    mt = np.einsum("pi,pi,pid->pd", Wi, K0, ut)
    ms = np.einsum("pi,pid->pd", Wi, K1)
    mts = np.einsum("pi,pid,pid->p", Wi, ut, K1)
    return m0, mt, ms, mts


def symmetric_singular_moments(geo: Geometry, k, t, s):
    """The near-singular rule averaged over both orders of the pair."""
    a0, at, as_, ats = singular_moments(geo, k, t, s)
    b0, bt, bs, bts = singular_moments(geo, k, s, t)
    return 0.5 * (a0 + b0), 0.5 * (at + bs), 0.5 * (as_ + bt), 0.5 * (ats + bts)


def pair_moments(geo: Geometry, k, t, s, chunk=8000):
    """Moments for pair arrays (t test, s source) with the rule chosen by
    is_near_singular.  Returns m0 [P], mt [P,3], ms [P,3], mts [P] complex."""
    t = np.asarray(t, np.int64)
    s = np.asarray(s, np.int64)
    P = t.shape[0]
    m0 = np.zeros(P, np.complex128)
    mt = np.zeros((P, 3), np.complex128)
    ms = np.zeros((P, 3), np.complex128)
    mts = np.zeros(P, np.complex128)
    near = is_near_singular(geo.cent, geo.h2, t, s)
    for mask, rule in ((near, symmetric_singular_moments), (~near, regular_moments)):
        idx = np.nonzero(mask)[0]
        for a in range(0, idx.size, chunk):
            sl = idx[a:a + chunk]
            r = rule(geo, k, t[sl], s[sl])
            m0[sl], mt[sl], ms[sl], mts[sl] = r
    return m0, mt, ms, mts
