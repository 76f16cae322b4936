"""Scattered field near the surface (Section 2) from the solution of the
PIEs and the charge density: the plain sum over quadrature points.

TEST INFRASTRUCTURE: imported only by tests/, never by the library.

Section 2 gives the near-zone field through the charge density
rho = i w eps0 n'.A - eps0 n'.grad'Phi.  With J and rho on the surface,

    E_s(r) = i w mu0 int_S J(r') g(r, r') dr' - (1/eps0) int_S rho(r') grad g(r, r') dr',

grad taken at the observation point r: grad g = (i k0 - 1/R) g (r - r') / R.
Reading (the paper names no rule): every triangle is integrated with the
7-point degree-5 rule, J|_t = a_t (r' - c_t) + beta_t from the RWG
coefficients, rho constant per triangle (pulse coefficients); accurate for
points farther than about a triangle size.

Pinned in tests/test_oracle_nearzone.py against closed forms: the Coulomb
field of a uniformly charged sphere outside it (Gauss's law), the field of
a small charged triangle far away, and the vector-potential field of a
small uniform current far away.
"""
import numpy as np

from . import constants as C
from .mesh import Topology, local_coefficients
from .quadrature import physical_points, radon7


def scattered_field(top: Topology, k0, x, rho, pts):
    """E_s at points pts [M,3] (complex [M,3]); x: PIE solution (mesh order,
    [E RWG ; T pulse], only the RWG part is used), rho: charge density per
    triangle (mesh order)."""
    w = C.omega_of_k(k0)
    b7, w7 = radon7()
    Q = physical_points(top.xyz, top.tri, b7)            # [T,7,3]
    W = w7[None, :] * top.area[:, None]                  # [T,7]
    a, beta, _ = local_coefficients(top, x)
    J = a[:, None, None] * (Q - top.centroid[:, None, :]) + beta[:, None, :]   # [T,7,3]
    rho = np.asarray(rho, np.complex128)
    pts = np.asarray(pts, np.float64)
    out = np.zeros((pts.shape[0], 3), np.complex128)
    for i, p in enumerate(pts):
        d = p[None, None, :] - Q                         # [T,7,3]
        R = np.linalg.norm(d, axis=2)
        g = np.exp(1j * k0 * R) / (4 * np.pi * R)
        gg = ((1j * k0 - 1.0 / R) * g / R)[..., None] * d
        out[i] = (1j * w * C.MU0 * np.einsum("tq,tq,tqd->d", W, g, J)
                  - (1.0 / C.EPS0) * np.einsum("tq,t,tqd->d", W, rho, gg))
    return out
