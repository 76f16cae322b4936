"""Adjoint products and gradients of far-field objectives (differentiation
through an adjoint GMRES solve), on the 1280-triangle sphere at kR = 0.01."""
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


def test_adjoint_identities(setup):
    import torch
    pg, xyz, tri, pr = setup
    u = torch.from_numpy(pi.complex_normal(pr.N, 1)).cuda()
    v = torch.from_numpy(pi.complex_normal(pr.N, 2)).cuda()
    lhs = torch.vdot(u, pr.apply(v)).item()
    rhs = torch.vdot(pr.apply_t(u, conj=True), v).item()
    # far-part rounding makes Z^T equal Z only to ~1e-5
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    t1 = torch.dot(u, pr.apply(v)).item()
    t2 = torch.dot(pr.apply_t(u), v).item()
    assert abs(t1 - t2) <= 1e-4 * abs(t1)
    rh = pi.bistatic_directions(37)
    Ep = torch.from_numpy(pi.complex_normal((37, 3), 3)).cuda()
    a = torch.vdot(Ep.reshape(-1), pr.farfield(v, rh).reshape(-1)).item()
    b = torch.vdot(pr.farfield_adjoint(Ep, rh), v).item()
    assert abs(a - b) <= 1e-12 * abs(a)


def excitations(pr):
    dirs = [([0, 0, -1.0], [1.0, 0, 0]), ([0, 0, -1.0], [0, 1.0, 0]),
            ([1.0, 0, 0], [0, 0, 1.0]), ([0, 1.0, 0], [1.0, 0, 0])]
    return dirs


def test_far_field_power_gradient(setup):
    """P(c) = sum_d |E_d(x(c))|^2, x = Z^-1 sum_j c_j b_j: the autograd gradient
    (adjoint solve) against central differences of the same GPU objective and
    against the oracle's exact gradient 2 G c, G = E^H E from dense solutions."""
    import torch

    from oracle.dense import assemble
    from oracle.excitation import rhs_planewave
    from oracle.farfield import far_field
    from oracle.mesh import build_topology
    import paper_1806_04164_gb300.autograd as pa

    pg, xyz, tri, pr = setup
    rh = pi.bistatic_directions(181)
    B = torch.stack([pr.rhs_planewave(k, e) for k, e in excitations(pr)], dim=1)  # [N, 4]
    c0 = torch.from_numpy(pi.complex_normal(4, 7)).cuda()

    def objective(c):
        x = pa.solve(pr, B @ c, tol=1e-5)
        E = pa.farfield(pr, x, rh)
        return (E.abs() ** 2).sum()

    c = c0.clone().requires_grad_(True)
    P = objective(c)
    P.backward()
    g = c.grad.detach().cpu().numpy()
    # central differences of the GPU objective (P is quadratic in c)
    fd = np.zeros(4, complex)
    with torch.no_grad():
        for j in range(4):
            h = 1e-2 * abs(c0[j].item())
            for unit, part in ((1.0, "re"), (1j, "im")):
                e = torch.zeros(4, dtype=c0.dtype, device="cuda")
                e[j] = unit * h
                d = (objective(c0 + e) - objective(c0 - e)).item() / (2 * h)
                fd[j] += d if part == "re" else 1j * d
    assert np.linalg.norm(g - fd) <= 1e-2 * np.linalg.norm(fd)
    # oracle: dense solutions of the four excitations
    top = build_topology(xyz, tri)
    Z = assemble(top, K)
    Bo = np.stack([rhs_planewave(top, K, k, e) for k, e in excitations(pr)], axis=1)
    X = np.linalg.solve(Z, Bo)
    Ej = np.stack([far_field(top, K, X[:, j], rh).reshape(-1) for j in range(4)], axis=1)
    G = Ej.conj().T @ Ej
    go = 2 * G @ c0.cpu().numpy()
    assert np.linalg.norm(g - go) <= 1e-2 * np.linalg.norm(go)
    print("gradient: vs FD", np.linalg.norm(g - fd) / np.linalg.norm(fd), "vs oracle",
          np.linalg.norm(g - go) / np.linalg.norm(go))
