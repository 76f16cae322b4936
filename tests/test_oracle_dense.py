"""Pins for oracle.dense (Galerkin matrix of Eqs. (1)-(2)) and for the whole
formulation against the Mie series (Section 4)."""
import numpy as np
import pytest

import pie_inputs as pi
from oracle import constants as C
from oracle import mie
from oracle.dense import assemble, rows
from oracle.excitation import rhs_planewave
from oracle.farfield import far_field, rcs
from oracle.mesh import build_topology, rwg_div, rwg_values
from oracle.moments import Geometry, is_near_singular
from oracle.quadrature import physical_points, radon7


@pytest.fixture(scope="module")
def small():
    xyz, tri = pi.icosphere(1)
    top = build_topology(xyz, tri)
    return top, assemble(top, 0.5)


def test_complex_symmetric(small):
    """Reciprocity: Z^T = Z to rounding in every block (regular pairs by the
    symmetric product rule, near-singular pairs by the two-sided average)."""
    top, Z = small
    E = top.E
    for blk in [(slice(0, E), slice(0, E)), (slice(E, None), slice(E, None)), (slice(0, E), slice(E, None))]:
        A = Z[blk]
        B = Z[blk[1], blk[0]].T
        assert np.abs(A - B).max() <= 1e-13 * np.abs(A).max()


def test_regular_entries_against_basis_values(small):
    """Independent assembly of the regular-pair part straight from RWG values
    at the quadrature points (no per-triangle moments)."""
    top, Z = small
    k = 0.5
    w = C.omega_of_k(k)
    geo = Geometry(top.xyz, top.tri)
    b7, w7 = radon7()
    P = physical_points(top.xyz, top.tri, b7)
    E = top.E
    rng = np.random.default_rng(3)
    checked = 0
    for _ in range(200):
        m, n = rng.integers(0, E, 2)
        tm, tn = top.edge_tri[m], top.edge_tri[n]
        pairs = [(t, s) for t in tm for s in tn]
        if any(is_near_singular(geo.cent, geo.h2, np.array([t]), np.array([s]))[0] for t, s in pairs):
            continue
        val = 0j
        for t, s in pairs:
            R = np.linalg.norm(P[t][:, None] - P[s][None], axis=-1)
            g = np.exp(1j * k * R) / (4 * np.pi * R)
            ft = rwg_values(top, m, t, P[t])
            fs = rwg_values(top, n, s, P[s])
            val += C.MU0 * np.einsum("i,j,id,jd,ij->", w7 * top.area[t], w7 * top.area[s], ft, fs, g)
        assert abs(Z[m, n] - val) <= 1e-12 * abs(val) + 1e-12 * np.abs(Z[:E, :E]).max()
        # pulse test (triangle t of m) against RWG n, and pulse-pulse
        t = tm[0]

        def I(t, s):
            R = np.linalg.norm(P[t][:, None] - P[s][None], axis=-1)
            g = np.exp(1j * k * R) / (4 * np.pi * R)
            return np.einsum("i,j,ij->", w7 * top.area[t], w7 * top.area[s], g)

        terms = [rwg_div(top, n, s) * I(t, s) for s in tn]
        ref = sum(terms)
        assert abs(Z[E + t, n] - ref) <= 1e-12 * sum(abs(v) for v in terms)
        assert abs(Z[E + t, E + tn[0]] - w * w * C.EPS0 * I(t, tn[0])) <= 1e-12 * abs(Z[E + t, E + tn[0]])
        checked += 1
    assert checked > 20


def test_rows_match_matrix(small):
    top, Z = small
    x = pi.complex_normal(top.N, 11)
    which = [0, 7, top.E - 1, top.E, top.N - 1]
    assert np.allclose(rows(top, 0.5, which, x), (Z @ x)[which], rtol=1e-12)


@pytest.mark.slow
def test_sphere_rcs_matches_mie():
    """PEC sphere R = 1 m, kR = 0.01, 1280 triangles, x-polarised plane wave
    along -z: bistatic RCS on the x-z (E-) plane within 0.1 dB of the Mie
    series wherever Mie is within 20 dB of its maximum."""
    k = 0.01
    xyz, tri = pi.icosphere(3)
    top = build_topology(xyz, tri)
    Z = assemble(top, k)
    b = rhs_planewave(top, k, [0, 0, -1], [1, 0, 0])
    x = np.linalg.solve(Z, b)
    rh = pi.bistatic_directions(181)
    s = rcs(far_field(top, k, x, rh))
    sm = mie.rcs_eplane(k, 1.0, -rh[:, 2])
    mask = sm > sm.max() * 1e-2
    db = np.abs(10 * np.log10(s[mask] / sm[mask]))
    assert db.max() < 0.1
    # the E-plane null (scattering angle 60 deg) is resolved
    assert 10 * np.log10(s[120] / s.max()) < -60


def test_rows_with_pair_mask_match_masked_matrix(small):
    top, _ = small
    c = top.centroid

    def mask(t, s):
        return np.linalg.norm(c[s] - c[t], axis=-1) < 0.6

    Zn = assemble(top, 0.5, pair_mask=lambda t, s: mask(t, s[None, :] if np.ndim(s) == 0 else s)
                  if np.ndim(t) == 0 else np.linalg.norm(c[s] - c[t], axis=-1) < 0.6)
    x = pi.complex_normal(top.N, 12)
    which = [1, 40, top.E + 3, top.N - 2]
    assert np.allclose(rows(top, 0.5, which, x, pair_mask=mask), (Zn @ x)[which], rtol=1e-12)


@pytest.mark.slow
def test_low_frequency_stability():
    """The PIEs stay stable as k -> 0 (Section 2): on a 320-triangle sphere
    the solved current scales as k (sigma / k^4 is the same to 1e-6 from
    kR = 1e-2 down to 1e-8, where an EFIE-type system breaks down) and the
    E-plane RCS keeps its distance from the Rayleigh limit."""
    xyz, tri = pi.icosphere(2)
    top = build_topology(xyz, tri)
    rh = pi.bistatic_directions(37)
    norm = []
    for k in (1e-2, 1e-4, 1e-6, 1e-8):
        Z = assemble(top, k)
        x = np.linalg.solve(Z, rhs_planewave(top, k, [0, 0, -1], [1, 0, 0]))
        s = rcs(far_field(top, k, x, rh))
        norm.append(s / k ** 4)
        sm = mie.rcs_eplane(k, 1.0, -rh[:, 2])
        mask = sm > sm.max() * 1e-2
        assert np.max(np.abs(10 * np.log10(s[mask] / sm[mask]))) < 0.35   # coarse mesh: 0.30 dB
    for v in norm[1:]:
        assert np.max(np.abs(v - norm[-1])) <= 1e-6 * np.max(norm[-1])
    assert np.max(np.abs(norm[0] - norm[-1])) <= 1e-3 * np.max(norm[-1])   # O((kR)^2) at kR = 1e-2


def test_rows_over_source_subsets_add_up(small):
    """rows(..., sources=S) is the partial sum over S: two halves give the row."""
    top, _ = small
    x = pi.complex_normal(top.N, 9)
    which = [0, 3, top.E, top.N - 1]
    full = rows(top, 0.3, which, x)
    half = np.arange(top.T) < top.T // 2
    a = rows(top, 0.3, which, x, sources=np.nonzero(half)[0])
    b = rows(top, 0.3, which, x, sources=np.nonzero(~half)[0])
    assert np.allclose(a + b, full, rtol=1e-12, atol=0)
