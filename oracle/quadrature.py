"""Triangle quadrature rules used by the Galerkin testing of Section 2.

The paper does not name its rules (reading: a 7-point degree-5 rule for all
regular integrals and a 64-point rule for the outer integral of near-singular
pairs).  Both rules are written here from their closed forms:

* ``radon7``: Radon (1948) 7-point rule, exact for total degree <= 5.  Points
  (1/3,1/3,1/3) with weight 9/40; the orbits of (a,a,1-2a) with
  a = (6 -+ sqrt15)/21 and weights (155 -+ sqrt15)/1200.
* ``collapsed_gauss(n)``: Gauss-Legendre in (u, v) on the unit square, mapped
  to the triangle by x = u, y = (1-u) v with Jacobian (1-u); exact for total
  degree <= 2n-2.

Weights are normalised to sum to 1, so a physical rule on triangle t has
weights w * area(t).  Pinned in tests/test_oracle_quadrature.py by monomial
integrals against the closed form a! b! / (a+b+2)!.
"""
import numpy as np


def radon7():
    """Barycentric coordinates [7,3] (weights of v0, v1, v2) and weights [7]."""
    s15 = np.sqrt(15.0)
    a1 = (6.0 - s15) / 21.0
    a2 = (6.0 + s15) / 21.0
    w1 = (155.0 - s15) / 1200.0
    w2 = (155.0 + s15) / 1200.0
    pts = [(1 / 3, 1 / 3, 1 / 3)]
    wts = [9.0 / 40.0]
    for a, w in ((a1, w1), (a2, w2)):
        b = 1.0 - 2.0 * a
        pts += [(b, a, a), (a, b, a), (a, a, b)]
        wts += [w, w, w]
    return np.array(pts, dtype=np.float64), np.array(wts, dtype=np.float64)


def gauss_legendre01(n: int):
    """n-point Gauss-Legendre nodes and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def collapsed_gauss(n: int):
    """n*n-point collapsed Gauss rule on the triangle, barycentric [n*n,3]
    and weights [n*n] summing to 1."""
    u, wu = gauss_legendre01(n)
    v, wv = gauss_legendre01(n)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            x = u[i]
            y = (1.0 - u[i]) * v[j]
            pts.append((1.0 - x - y, x, y))
            wts.append(2.0 * wu[i] * wv[j] * (1.0 - u[i]))
    return np.array(pts, dtype=np.float64), np.array(wts, dtype=np.float64)


def physical_points(xyz, tri, bary):
    """Quadrature points of every triangle: [T, Q, 3]."""
    v0 = xyz[tri[:, 0]]
    v1 = xyz[tri[:, 1]]
    v2 = xyz[tri[:, 2]]
    return (bary[None, :, 0, None] * v0[:, None, :]
            + bary[None, :, 1, None] * v1[:, None, :]
            + bary[None, :, 2, None] * v2[:, None, :])
