"""Pins for oracle.mesh (RWG / pulse discretisation, Section 2)."""
import numpy as np
import pytest

import pie_inputs as pi
from oracle.mesh import build_topology, local_coefficients, rwg_div, rwg_values
from oracle.quadrature import physical_points, radon7


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_icosphere_counts_and_euler(n):
    xyz, tri = pi.icosphere(n)
    top = build_topology(xyz, tri)
    assert top.T == 20 * 4 ** n and top.E == 30 * 4 ** n and xyz.shape[0] == 10 * 4 ** n + 2
    assert xyz.shape[0] - top.E + top.T == 2
    assert np.all(top.edges[:, 0] < top.edges[:, 1])
    assert np.all(np.diff(top.edges[:, 0] * 10 ** 7 + top.edges[:, 1]) > 0)


def test_rwg_identity_and_continuity():
    """int f_n dS = - int r div f_n dS (surface divergence theorem; fixes the
    sign of f against its divergence) and continuity of the normal component
    of f_n across its edge."""
    xyz, tri = pi.icosphere(1)
    top = build_topology(xyz, tri)
    b7, w7 = radon7()
    P = physical_points(top.xyz, top.tri, b7)
    for n in range(top.E):
        lhs = np.zeros(3)
        rhs = np.zeros(3)
        for t in top.edge_tri[n]:
            W = w7 * top.area[t]
            lhs += np.sum(W[:, None] * rwg_values(top, n, t, P[t]), axis=0)
            rhs -= rwg_div(top, n, t) * np.sum(W[:, None] * P[t], axis=0)
        assert np.allclose(lhs, rhs, atol=1e-14)
        a, b = top.xyz[top.edges[n]]
        mid = 0.5 * (a + b)
        tp, tm = top.edge_tri[n]
        e = (b - a) / np.linalg.norm(b - a)
        mp = np.cross(e, top.normal[tp])
        mp = mp if np.dot(mp, top.centroid[tp] - mid) < 0 else -mp   # outward from T+
        mm = np.cross(e, top.normal[tm])
        mm = mm if np.dot(mm, top.centroid[tm] - mid) > 0 else -mm   # into T-
        fp = rwg_values(top, n, tp, mid)
        fm = rwg_values(top, n, tm, mid)
        assert abs(np.dot(fp, mp) - 1.0) < 1e-12 and abs(np.dot(fm, mm) - 1.0) < 1e-12


def test_local_coefficients_reproduce_rwg_sum():
    xyz, tri = pi.icosphere(1)
    top = build_topology(xyz, tri)
    x = pi.complex_normal(top.N, 5)
    a, beta, sig = local_coefficients(top, x)
    b7, _ = radon7()
    P = physical_points(top.xyz, top.tri, b7)
    for t in range(top.T):
        J = sum(x[n] * rwg_values(top, n, t, P[t]) for n in top.tri_edges[t])
        J2 = a[t] * (P[t] - top.centroid[t]) + beta[t]
        assert np.allclose(J, J2, atol=1e-12)
        div = sum(x[n] * rwg_div(top, n, t) for n in top.tri_edges[t])
        assert abs(div - 2 * a[t]) < 1e-10


def test_rejects_nonmanifold_and_degenerate():
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, -1, 0.5]], float)
    with pytest.raises(ValueError):
        build_topology(xyz, np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]]))
    with pytest.raises(ValueError):
        build_topology(np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0.]]), np.array([[0, 1, 2]]))
