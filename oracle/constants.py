"""Free-space constants (Section 2: PEC objects in free space, exp(-i w t)).

Reading: mu0 = 4*pi*1e-7 H/m exactly, c0 = 299792458 m/s, eps0 = 1/(mu0 c0^2),
k0 = w sqrt(mu0 eps0) = w / c0.
"""
import math

MU0 = 4.0e-7 * math.pi
C0 = 299792458.0
EPS0 = 1.0 / (MU0 * C0 * C0)


def omega_of_k(k0: float) -> float:
    """Angular frequency for wavenumber k0 (Section 2: k0 = w sqrt(mu0 eps0))."""
    return k0 * C0
