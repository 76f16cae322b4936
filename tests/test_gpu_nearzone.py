"""Near-zone fields through Eq. (3) (Section 2) on the 1280-triangle PEC
sphere at kR = 0.01: the single-layer operator against the oracle's dense
pulse-pulse block, the charge density against the quasi-static surface
charge of a conducting sphere in a uniform field (3 eps0 E0 x / R), and the
extinction of the total field inside the conductor."""
import numpy as np
import pytest

import pie_inputs as pi

pytestmark = pytest.mark.gpu
K = 0.01


@pytest.fixture(scope="module")
def setup():
    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    xyz, tri = pi.icosphere(3)
    return pg, xyz, tri, pg.Problem(pg.Mesh(xyz, tri), K, 3, root_side=2.0)


def test_single_layer_matches_dense_block(setup):
    import torch
    from oracle import constants as C
    from oracle.dense import assemble
    from oracle.mesh import build_topology
    pg, xyz, tri, pr = setup
    top = build_topology(xyz, tri)
    Z = assemble(top, K)
    w2e = C.omega_of_k(K) ** 2 * C.EPS0
    S = Z[top.E:, top.E:] / w2e
    q = pi.complex_normal(top.T, 4)
    y = pr.apply_single_layer(torch.from_numpy(q).cuda()).cpu().numpy()
    assert np.linalg.norm(y - S @ q) <= 1e-3 * np.linalg.norm(S @ q)


def test_charge_density_and_interior_extinction(setup):
    import torch
    from oracle import constants as C
    pg, xyz, tri, pr = setup
    kh, pol = [0, 0, -1.0], [1.0, 0, 0]
    b = pr.rhs_planewave(kh, pol)
    x, st = pr.solve(b, tol=1e-6, maxit=2000, restart=300)
    assert st["converged"]
    bq = pr.rhs_potential(kh, pol)
    dn, st2 = pr.solve_single_layer(bq, tol=1e-6)
    assert st2["converged"], st2
    w = C.omega_of_k(K)
    sigma = x[pr.E:]
    rho = 1j * w * C.EPS0 * sigma - C.EPS0 * dn
    v = xyz[tri]
    cx = v.mean(axis=1)[:, 0]
    ref = 3 * C.EPS0 * cx          # quasi-static, R = 1, E0 = 1
    r = rho.cpu().numpy()
    err = np.linalg.norm(r - ref) / np.linalg.norm(ref)
    print("charge density vs quasi-static:", err, "iterations", st2["iterations"])
    assert err < 3e-2
    # total field inside the conductor vanishes (incident field there: x-hat e^{-ikz})
    rng = np.random.default_rng(3)
    pts = rng.uniform(-0.4, 0.4, (20, 3))
    Es = pr.nearfield(x, rho, pts).cpu().numpy()
    Ei = np.exp(1j * K * (pts @ np.array(kh)))[:, None] * np.array(pol)[None, :]
    ext = np.max(np.linalg.norm(Es + Ei, axis=1))
    print("interior total field / E0:", ext)
    assert ext < 2e-2
    # outside: quasi-static dipole field E_s = -grad(E0 R^3 x / r^3), at r = 1.6 R
    pts = rng.normal(size=(20, 3))
    pts *= 1.6 / np.linalg.norm(pts, axis=1, keepdims=True)
    Es = pr.nearfield(x, rho, pts).cpu().numpy()
    rr = np.linalg.norm(pts, axis=1)
    ex = np.zeros_like(pts)
    ex[:, 0] = 1.0
    dip = -(ex / rr[:, None] ** 3 - 3 * pts[:, :1] * pts / rr[:, None] ** 5)
    dev = np.max(np.linalg.norm(Es - dip, axis=1)) / np.max(np.linalg.norm(dip, axis=1))
    print("exterior scattered field vs quasi-static dipole:", dev)
    assert dev < 3e-2


def test_nearfield_matches_oracle_sum(setup):
    """pie_nearfield against oracle.nearzone's plain sum over the same
    quadrature points, for a random current and charge density, at points
    from 0.3 to 1 m off the surface: equal to rounding."""
    import torch
    from oracle.mesh import build_topology
    from oracle.nearzone import scattered_field
    pg, xyz, tri, pr = setup
    top = build_topology(xyz, tri)
    x = pi.complex_normal(pr.N, 41)
    rho = pi.complex_normal(pr.T, 42)
    rng = np.random.default_rng(3)
    d = rng.normal(size=(12, 3))
    pts = d / np.linalg.norm(d, axis=1)[:, None] * rng.uniform(1.3, 2.0, size=(12, 1))
    E = pr.nearfield(torch.from_numpy(x).cuda(), torch.from_numpy(rho).cuda(), pts).cpu().numpy()
    Eo = scattered_field(top, K, x, rho, pts)
    assert np.linalg.norm(E - Eo) <= 1e-10 * np.linalg.norm(Eo)
