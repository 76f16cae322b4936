"""Right-hand sides for general incident potentials (pie_rhs_potentials at
the points of pie_problem_quadrature), and several columns in one solve /
far-field call, against the oracle and against one-column calls."""
import numpy as np
import pytest

import pie_inputs as pi

pytestmark = pytest.mark.gpu

K = 0.01


@pytest.fixture(scope="module")
def pg():
    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    return pg


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def dipole_potentials(P, k0, r0, p):
    """Potentials of a small oscillating source at r0 (any smooth, non-plane
    field serves here): Phi = exp(i k R)/R, A = p exp(i k R)/R."""
    R = np.linalg.norm(P - r0, axis=-1)
    g = np.exp(1j * k0 * R) / R
    return g[..., None] * p, g


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_rhs_potentials_match_oracle_and_planewave(pg, prec):
    import torch
    from oracle.excitation import potentials, quadrature_points, rhs_from_potentials
    from oracle.mesh import build_topology
    xyz, tri = pi.icosphere(3)
    top = build_topology(xyz, tri)
    pr = pg.Problem(pg.Mesh(xyz, tri), K, 4, root_side=2.0, precision=prec)
    pts, wts = pr.quadrature()
    Po, Wo = quadrature_points(top)
    assert np.allclose(pts, Po, rtol=0, atol=1e-15) and np.allclose(wts, Wo, rtol=1e-14, atol=0)
    tol = 1e-6 if prec == 1 else 1e-13
    # a plane wave through the general call is the plane-wave call
    kh, pol = np.array([0.0, 0.6, -0.8]), np.array([1.0, 0.0, 0.0])
    A, Phi = potentials(pts, K, kh, pol)
    b = pr.rhs_potentials(torch.from_numpy(A).cuda(), torch.from_numpy(Phi).cuda()).cpu().numpy()
    assert rel(b, pr.rhs_planewave(kh, pol).cpu().numpy()) < tol
    # a non-plane field against the oracle
    A, Phi = dipole_potentials(pts, K, np.array([0.1, -0.2, 3.0]), np.array([0.3, 1.0, -0.5]))
    b = pr.rhs_potentials(torch.from_numpy(A).cuda(), torch.from_numpy(Phi).cuda()).cpu().numpy()
    bo = rhs_from_potentials(top, K, A, Phi)
    for sl in (slice(0, top.E), slice(top.E, None)):
        assert rel(b[sl], bo[sl]) < tol


def test_solve_and_farfield_columns(pg):
    """Two plane waves in one pie_solve / pie_farfield call equal the
    one-column calls bit for bit (the columns are solved one after another
    by the same code)."""
    import torch
    pr = pg.Problem(pg.Mesh(*pi.icosphere(3)), K, 4, root_side=2.0, precision=pg.PIE_MIXED)
    B = torch.stack([pr.rhs_planewave([0, 0, -1.0], [1.0, 0, 0]), pr.rhs_planewave([0, 0, -1.0], [0, 1.0, 0])])
    X, stats = pr.solve(B, tol=1e-6, maxit=2000, restart=100)
    assert len(stats) == 2 and all(s["converged"] for s in stats)
    rh = pi.bistatic_directions(19)
    E = pr.farfield(X, rh)
    assert E.shape == (2, 19, 3)
    for j in range(2):
        x, st = pr.solve(B[j].contiguous(), tol=1e-6, maxit=2000, restart=100)
        assert torch.equal(X[j], x) and st["iterations"] == stats[j]["iterations"]
        assert torch.equal(E[j], pr.farfield(x, rh))


def test_rhs_potential_of_eq3_matches_oracle(pg):
    """pie_rhs_potential, the right-hand side <p_t, Phi^inc> of Eq. (3), is
    the pulse part of the PIE right-hand side divided by -i w eps0."""
    from oracle import constants as C
    from oracle.excitation import rhs_planewave
    from oracle.mesh import build_topology
    xyz, tri = pi.icosphere(3)
    top = build_topology(xyz, tri)
    pr = pg.Problem(pg.Mesh(xyz, tri), K, 3, root_side=2.0, precision=pg.PIE_FP64)
    kh, pol = [0.6, 0.0, -0.8], [0.8, 0.0, 0.6]
    bq = pr.rhs_potential(kh, pol).cpu().numpy()
    bo = rhs_planewave(top, K, kh, pol)[top.E:] / (-1j * C.omega_of_k(K) * C.EPS0)
    assert rel(bq, bo) < 1e-12
