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
