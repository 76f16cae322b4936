"""Pins for oracle.quadrature: monomial integrals over the reference triangle
(0,0),(1,0),(0,1) against the closed form a! b! / (a+b+2)!."""
from math import factorial

import numpy as np

from oracle.quadrature import collapsed_gauss, radon7


def exact(a, b):
    return factorial(a) * factorial(b) / factorial(a + b + 2)


def integrate(rule, a, b):
    bary, w = rule
    x, y = bary[:, 1], bary[:, 2]
    return 0.5 * np.sum(w * x ** a * y ** b)   # area 1/2, weights sum to 1


def test_radon7_degree5_exact_and_not_degree6():
    r = radon7()
    assert abs(r[1].sum() - 1) < 1e-15
    for a in range(6):
        for b in range(6 - a):
            assert abs(integrate(r, a, b) - exact(a, b)) < 1e-15
    worst = max(abs(integrate(r, a, 6 - a) - exact(a, 6 - a)) for a in range(7))
    assert worst > 1e-6


def test_collapsed_gauss_degree():
    for n in (4, 8):
        r = collapsed_gauss(n)
        assert abs(r[1].sum() - 1) < 1e-14
        for a in range(2 * n - 1):
            for b in range(2 * n - 1 - a):
                assert abs(integrate(r, a, b) - exact(a, b)) < 1e-15
