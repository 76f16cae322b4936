"""Pins for oracle.singular: closed-form potential integrals against
brute-force Gauss integration (no closed forms on the reference side)."""
import numpy as np
import pytest

from oracle.quadrature import collapsed_gauss
from oracle.singular import potential_integrals
from tests._reference_integrals import inner_reference

V = np.array([[0.0, 0.0, 0.0], [1.0, 0.2, 0.0], [0.3, 0.9, 0.1]])


def brute(r):
    # static kernel: k = 0
    I0, I1 = inner_reference(r, V, 0.0, n=60)
    c = V.mean(axis=0)
    # inner_reference returns moments about the centroid; convert to (r'-r)
    return 4 * np.pi * I0.real, 4 * np.pi * (I1.real + (c - r) * I0.real)


@pytest.mark.parametrize("r", [
    [0.4, 0.3, 0.5], [2.0, 1.0, 0.3], [0.4, 0.3, 0.2], [-0.5, -0.4, -0.3],
])
def test_offplane(r):
    r = np.array(r)
    I1, Ir = potential_integrals(r, *V)
    b1, br = brute(r)
    assert abs(I1 - b1) < 1e-10 * abs(b1)
    assert np.allclose(Ir, br, rtol=0, atol=1e-10 * np.linalg.norm(br))


@pytest.mark.parametrize("bc", [
    (0.2, 0.5, 0.3), (0.0, 0.5, 0.5), (1.0, 0.0, 0.0), (-0.2, 0.6, 0.6), (0.5, 0.5, 0.0), (1.5, -0.3, -0.2),
])
def test_inplane_including_edges_vertices_and_outside(bc):
    r = bc[0] * V[0] + bc[1] * V[1] + bc[2] * V[2]
    I1, Ir = potential_integrals(r, *V)
    b1, br = brute(r)
    assert abs(I1 - b1) < 1e-11 * abs(b1)
    assert np.allclose(Ir, br, rtol=0, atol=1e-11 * np.linalg.norm(br))


def test_sheet_jump():
    """Normal derivative of the single-layer potential of a uniform sheet jumps
    by 4 pi across it: I1(d) ~ I1(0) - 2 pi |d| near an interior point."""
    c = V.mean(axis=0)
    n = np.cross(V[1] - V[0], V[2] - V[0])
    n /= np.linalg.norm(n)
    d = 1e-6
    up = potential_integrals(c + d * n, *V)[0]
    dn = potential_integrals(c - d * n, *V)[0]
    mid = potential_integrals(c, *V)[0]
    assert abs((up - mid) / d + 2 * np.pi) < 1e-4
    assert abs((dn - mid) / d + 2 * np.pi) < 1e-4
