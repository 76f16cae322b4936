"""Incident potentials and the right-hand side of Eqs. (1)-(2).

The paper gives the PIE right-hand sides in terms of A^inc and Phi^inc
(Section 2) but not the gauge used for a plane wave.  Reading: for
E^inc = e E0 exp(i k khat.r) (e . khat = 0) take the Lorenz-gauge pair that
stays finite as k -> 0,

  Phi^inc = -E0 (e.r) exp(i k khat.r),   A^inc = -(E0/c0) (e.r) khat exp(i k khat.r),

which satisfies E = i w A - grad Phi, div A = i w mu0 eps0 Phi and the
Helmholtz equation (checked by finite differences in
tests/test_oracle_excitation.py).  Right-hand side, tested as the operator:

  b_J[m] = -<f_m, A^inc>,   b_sigma[t] = -i w eps0 <p_t, Phi^inc>,

integrated with the 7-point rule.
"""
import numpy as np

from . import constants as C
from .mesh import Topology
from .quadrature import physical_points, radon7


def potentials(r, k0, khat, pol, E0=1.0):
    """(A [...,3], Phi [...]) of the plane wave at points r [...,3]."""
    r = np.asarray(r, np.float64)
    khat = np.asarray(khat, np.float64)
    pol = np.asarray(pol, np.float64)
    ph = np.exp(1j * k0 * (r @ khat))
    er = r @ pol
    Phi = -E0 * er * ph
    A = (-(E0 / C.C0) * er * ph)[..., None] * khat
    return A, Phi


def quadrature_points(top: Topology):
    """Points [T,7,3] and weights [T,7] (area included) of the 7-point rule."""
    b7, w7 = radon7()
    return physical_points(top.xyz, top.tri, b7), w7[None, :] * top.area[:, None]


def rhs_planewave(top: Topology, k0, khat, pol, E0=1.0):
    """b in mesh order [E ; T] (complex128)."""
    P, _ = quadrature_points(top)
    A, Phi = potentials(P, k0, khat, pol, E0)
    return rhs_from_potentials(top, k0, A, Phi)


def rhs_from_potentials(top: Topology, k0, A, Phi):
    """b in mesh order for incident potentials given at the quadrature points
    of quadrature_points: A [T,7,3], Phi [T,7]."""
    P, W = quadrature_points(top)
    A = np.asarray(A, np.complex128)
    Phi = np.asarray(Phi, np.complex128)
    w = C.omega_of_k(k0)
    b = np.zeros(top.N, np.complex128)
    b[top.E:] = -1j * w * C.EPS0 * np.sum(W * Phi, axis=1)
    for t in range(top.T):
        for kk in range(3):
            n = top.tri_edges[t, kk]
            if n < 0:
                continue
            s = top.tri_sign[t, kk]
            p = top.xyz[top.edge_free[n, 0 if s > 0 else 1]]
            f = s * top.edge_len[n] / (2.0 * top.area[t]) * (P[t] - p)   # [7,3]
            b[n] += -np.sum(W[t][:, None] * f * A[t])
    return b
