"""Pins for oracle.moments: the near-singular rule against nested brute-force
Gauss integration on two-triangle meshes, and exact identities of the
regular rule."""
import numpy as np
import pytest

import pie_inputs as pi
from oracle.moments import (Geometry, is_near_singular, pair_moments, regular_moments, singular_moments,
                            symmetric_singular_moments)
from tests._reference_integrals import pair_reference


@pytest.mark.parametrize("shared", ["edge", "fold", "vertex"])
@pytest.mark.parametrize("order", [(0, 1), (1, 0), (0, 0)])
def test_singular_rule_against_brute_force(shared, order):
    xyz, tri = pi.flat_pair(shared)
    geo = Geometry(xyz, tri)
    t, s = order
    k = 2.0
    got = singular_moments(geo, k, np.array([t]), np.array([s]))
    ref = pair_reference(geo.v[t], geo.v[s], k)
    # error scale of each moment: |m0| h^j for a moment of polynomial degree j
    h = np.sqrt(max(geo.h2[t], geo.h2[s]))
    scales = [abs(ref[0]), abs(ref[0]) * h, abs(ref[0]) * h, abs(ref[0]) * h * h]
    for g, r, sc in zip(got, ref, scales):
        g = np.ravel(g)
        r = np.ravel(r)
        assert np.linalg.norm(g - r) <= 1e-3 * sc


def test_regular_rule_symmetry_and_static_limit():
    xyz, tri = pi.icosphere(1)
    geo = Geometry(xyz, tri)
    t = np.array([0, 3, 10, 40])
    s = np.array([60, 70, 79, 2])
    a = regular_moments(geo, 0.3, t, s)
    b = regular_moments(geo, 0.3, s, t)
    assert np.allclose(a[0], b[0], rtol=1e-14)
    assert np.allclose(a[3], b[3], rtol=1e-13)
    assert np.allclose(a[1], b[2], rtol=1e-13)
    # k -> 0: imaginary part -> k/(4 pi) * area_t * area_s, real part -> static
    k = 1e-6
    m0 = regular_moments(geo, k, t, s)[0]
    assert np.allclose(m0.imag, k / (4 * np.pi) * geo.area[t] * geo.area[s], rtol=1e-8)
    m00 = regular_moments(geo, 0.0, t, s)[0]
    assert np.allclose(m0.real, m00.real, rtol=1e-10)


def test_classification_is_local_and_symmetric():
    xyz, tri = pi.icosphere(2)
    geo = Geometry(xyz, tri)
    T = tri.shape[0]
    tt, ss = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    near = is_near_singular(geo.cent, geo.h2, tt.ravel(), ss.ravel()).reshape(T, T)
    assert np.array_equal(near, near.T)
    assert np.all(np.diag(near))
    # every pair sharing a vertex is near-singular
    for t in range(0, T, 7):
        for s in range(T):
            if set(tri[t]) & set(tri[s]):
                assert near[t, s]


def test_pair_moments_dispatch():
    xyz, tri = pi.icosphere(1)
    geo = Geometry(xyz, tri)
    t = np.array([0, 0, 5])
    s = np.array([0, 50, 5])
    m = pair_moments(geo, 0.1, t, s)
    near = is_near_singular(geo.cent, geo.h2, t, s)
    for i in range(3):
        rule = symmetric_singular_moments if near[i] else regular_moments
        r = rule(geo, 0.1, t[i:i + 1], s[i:i + 1])
        assert np.allclose(m[0][i], r[0][0]) and np.allclose(m[3][i], r[3][0])


def test_symmetrised_rule_is_reciprocal_and_accurate():
    """Both orders of the averaged rule give swapped moments exactly, and the
    average stays within the brute-force bar."""
    xyz, tri = pi.flat_pair("fold")
    geo = Geometry(xyz, tri)
    a = symmetric_singular_moments(geo, 2.0, np.array([0]), np.array([1]))
    b = symmetric_singular_moments(geo, 2.0, np.array([1]), np.array([0]))
    assert np.allclose(a[0], b[0], rtol=1e-15) and np.allclose(a[3], b[3], rtol=1e-15)
    assert np.allclose(a[1], b[2], rtol=1e-15) and np.allclose(a[2], b[1], rtol=1e-15)
    ref = pair_reference(geo.v[0], geo.v[1], 2.0)
    h = np.sqrt(max(geo.h2))
    for g, r, sc in zip(a, ref, [abs(ref[0]), abs(ref[0]) * h, abs(ref[0]) * h, abs(ref[0]) * h * h]):
        assert np.linalg.norm(np.ravel(g) - np.ravel(r)) <= 1e-3 * sc
