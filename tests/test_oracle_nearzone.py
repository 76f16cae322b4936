"""Pins for oracle.nearzone against closed forms of electrostatics and of a
small current element."""
import numpy as np

import pie_inputs as pi
from oracle import constants as C
from oracle.mesh import build_topology
from oracle.nearzone import scattered_field


def test_charged_sphere_is_a_point_charge_outside():
    """Uniform charge on a closed sphere, k -> 0: outside, E = Q r_hat /
    (4 pi eps0 r^2) (Gauss), at every distance; Q = rho x area."""
    xyz, tri = pi.icosphere(4)
    top = build_topology(xyz, tri)
    rho = np.full(top.T, 2.0 + 0.5j)
    Q = rho[0] * top.area.sum()
    pts = np.array([[0, 0, 1.5], [2.0, 1.0, -0.5], [0.3, -3.0, 0.2]])
    E = scattered_field(top, 1e-9, np.zeros(top.N), rho, pts)
    for p, e in zip(pts, E):
        r = np.linalg.norm(p)
        want = Q * p / (4 * np.pi * C.EPS0 * r ** 3)
        assert np.linalg.norm(e - want) <= 2e-4 * np.linalg.norm(want)


def test_small_charged_triangle_far_away():
    xyz, tri = pi.flat_pair("edge")
    top = build_topology(xyz * 1e-3, tri)                # millimetre triangles
    rho = np.array([1.0 + 0j, -0.25 + 0j])
    Q = np.sum(rho * top.area)
    c = np.sum(top.centroid * (rho * top.area)[:, None].real, axis=0) / Q.real
    p = np.array([0.3, -0.2, 0.5])
    E = scattered_field(top, 1e-9, np.zeros(top.N), rho, p[None])[0]
    d = p - c
    want = Q * d / (4 * np.pi * C.EPS0 * np.linalg.norm(d) ** 3)
    assert np.linalg.norm(E - want) <= 1e-5 * np.linalg.norm(want)


def test_small_uniform_current_far_away():
    """A uniform current density J0 on a small patch of area A: the first term
    alone, E = i w mu0 J0 A exp(i k R) / (4 pi R) (no charge)."""
    xyz, tri = pi.flat_pair("edge")
    top = build_topology(xyz * 1e-3, tri)
    k = 0.7
    # RWG coefficient of the shared edge scaled so that J is the RWG function
    x = np.zeros(top.N, np.complex128)
    x[0] = 1.0
    from oracle.mesh import local_coefficients
    a, beta, _ = local_coefficients(top, x)
    p = np.array([0.4, 0.1, 0.9])
    E = scattered_field(top, k, x, np.zeros(top.T), p[None])[0]
    want = np.zeros(3, np.complex128)
    w = C.omega_of_k(k)
    for t in range(top.T):
        # the affine J integrates to A_t beta_t over the triangle (a multiplies r - c_t)
        R = np.linalg.norm(p - top.centroid[t])
        want += 1j * w * C.MU0 * top.area[t] * beta[t] * np.exp(1j * k * R) / (4 * np.pi * R)
    assert np.linalg.norm(E - want) <= 1e-4 * np.linalg.norm(want)
