"""Far-zone scattered field from J alone (Section 2: for far-zone scattering J
is sufficient).

E_far(rhat) = i w mu0 / (4 pi) (I - rhat rhat) . sum_t int_t J(r') exp(-i k rhat.r') dr'
with the factor exp(i k r)/r removed; RCS = 4 pi |E_far|^2 / E0^2.  J on each
triangle is the affine restriction of the RWG expansion (oracle.mesh), the
integral uses the 7-point rule.
"""
import numpy as np

from . import constants as C
from .mesh import Topology, local_coefficients
from .quadrature import physical_points, radon7


def far_field(top: Topology, k0, x, rhat):
    rhat = np.asarray(rhat, np.float64)
    a, beta, _ = local_coefficients(top, x)
    b7, w7 = radon7()
    P = physical_points(top.xyz, top.tri, b7)            # [T,7,3]
    W = w7[None, :] * top.area[:, None]
    J = a[:, None, None] * (P - top.centroid[:, None, :]) + beta[:, None, :]   # [T,7,3]
    ph = np.exp(-1j * k0 * np.einsum("tqd,nd->ntq", P, rhat))                 # [n,T,7]
    F = np.einsum("ntq,tq,tqd->nd", ph, W, J)
    F = F - rhat * np.sum(rhat * F, axis=1, keepdims=True)
    w = C.omega_of_k(k0)
    return 1j * w * C.MU0 / (4.0 * np.pi) * F


def rcs(E, E0=1.0):
    return 4.0 * np.pi * np.sum(np.abs(E) ** 2, axis=-1) / (E0 * E0)
