import numpy as np

from oracle.gmres import gmres


def test_gmres_matches_direct_solve():
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) * 20 + rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for restart in (10, 100):
        x, it, hist = gmres(lambda v: A @ v, b, tol=1e-12, restart=restart)
        assert np.linalg.norm(x - np.linalg.solve(A, b)) < 1e-10 * np.linalg.norm(x)
        assert hist[-1] <= 1e-12
