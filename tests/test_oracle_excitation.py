"""Pins for the plane-wave gauge (reading of Section 2's A^inc, Phi^inc)."""
import numpy as np

from oracle import constants as C
from oracle.excitation import potentials


def grad(f, r, h=1e-4):
    out = []
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        out.append((f(r + e) - f(r - e)) / (2 * h))
    return np.stack(out, axis=-1)


def test_fields_gauge_helmholtz():
    k = 0.7
    w = C.omega_of_k(k)
    khat = np.array([0.3, -0.4, np.sqrt(1 - 0.25)])
    pol = np.cross(khat, [0, 0, 1.0])
    pol /= np.linalg.norm(pol)
    r = np.array([0.3, -0.2, 0.5])
    A, Phi = potentials(r, k, khat, pol)
    E = 1j * w * A - grad(lambda q: potentials(q, k, khat, pol)[1], r)
    Einc = pol * np.exp(1j * k * khat @ r)
    assert np.allclose(E, Einc, atol=1e-7)
    divA = sum(grad(lambda q, i=i: potentials(q, k, khat, pol)[0][i], r)[i] for i in range(3))
    assert abs(divA - 1j * w * C.MU0 * C.EPS0 * Phi) < 1e-7 * abs(divA)
    h = 1e-3
    lap = sum((potentials(r + h * e, k, khat, pol)[1] - 2 * Phi + potentials(r - h * e, k, khat, pol)[1]) / h ** 2
              for e in np.eye(3))
    assert abs(lap + k * k * Phi) < 1e-5


def test_rhs_from_potentials_closed_forms():
    """Constant and linear potentials, whose testing integrals the 7-point
    rule computes exactly: b_sigma = -i w eps0 A_t (phi0 + g.c_t) and
    b_J[m] = -a0 . int f_m = -a0 . (l_m / 2) [(c+ - p+) - (c- - p-)]."""
    import pie_inputs as pi
    from oracle.excitation import quadrature_points, rhs_from_potentials
    from oracle.mesh import build_topology
    xyz, tri = pi.icosphere(2)
    top = build_topology(xyz, tri)
    k0 = 0.3
    w = C.omega_of_k(k0)
    P, W = quadrature_points(top)
    assert np.allclose(W.sum(axis=1), top.area, rtol=1e-14, atol=0)
    a0 = np.array([0.2 - 0.1j, -0.7 + 0.3j, 0.4 + 0.0j])
    phi0, g = 1.3 - 0.2j, np.array([0.5, -0.25, 2.0])
    A = np.broadcast_to(a0, P.shape)
    Phi = phi0 + P @ g
    b = rhs_from_potentials(top, k0, A, Phi)
    want_s = -1j * w * C.EPS0 * top.area * (phi0 + top.centroid @ g)
    assert np.allclose(b[top.E:], want_s, rtol=1e-13, atol=0)
    want_J = np.zeros(top.E, np.complex128)
    for n in range(top.E):
        tp, tm = top.edge_tri[n]
        pp, pm = top.xyz[top.edge_free[n, 0]], top.xyz[top.edge_free[n, 1]]
        fint = 0.5 * top.edge_len[n] * ((top.centroid[tp] - pp) - (top.centroid[tm] - pm))
        want_J[n] = -a0 @ fint
    assert np.allclose(b[:top.E], want_J, rtol=1e-12, atol=1e-15 * np.abs(want_J).max())
