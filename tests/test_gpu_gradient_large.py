"""The differentiation workload at its stated size: the gradient of the
total scattered far-field power over 181 bistatic angles with respect to 64
complex excitation coefficients on the 81,920-triangle sphere at kR = 1e-3
(6-level MLFMA), through the adjoint of the nested solve.  The objective
P(c) = sum_d |E_d(Z^-1 sum_j c_j b_j)|^2 is a real quadratic form in c, so
central differences of the same GPU objective are exact for any step, up
to the solves' residuals; the step is |c_j| itself, so that those residuals
(1e-6 of each P) enter the difference quotient divided by a step of the
coefficient's own size.  torch's conjugate-Wirtinger gradient is
dP/da_j + i dP/db_j for c_j = a_j + i b_j.  The adjoint solve runs to 1e-4 (the receiving-type
right-hand side F^H E stalls near 2.5e-5 at this size); 1e-4 bounds the
gradient's relative error well below the 1e-3 of the check."""
import numpy as np
import pytest

import pie_inputs as pi

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_far_field_power_gradient_81920_triangles():
    import torch
    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    import paper_1806_04164_gb300.autograd as pa
    k0, L = 1e-3, 6
    mesh = pg.Mesh(*pi.icosphere(6))
    pr = pg.Problem(mesh, k0, L, root_side=2.0, precision=pg.PIE_MIXED)
    pin = pg.Problem(mesh, k0, L, root_side=2.0, precision=pg.PIE_FP32H, tau=3, kappa_a=0.15, ntheta=4)
    assert pr.T == 81920
    waves = pi.planewave_set()
    B = torch.stack([pr.rhs_planewave(k, e) for k, e in waves], dim=1)          # [N, 64]
    rh = pi.bistatic_directions(181)
    c0 = torch.from_numpy(pi.complex_normal(64, 7)).cuda()

    def objective(c):
        x = pa.solve(pr, B @ c, tol=1e-6, adj_tol=1e-4, inner=pin)
        return (pa.farfield(pr, x, rh).abs() ** 2).sum()

    c = c0.clone().requires_grad_(True)
    P = objective(c)
    P.backward()
    g = c.grad.detach().cpu().numpy()
    assert g.shape == (64,) and np.all(np.isfinite(g))
    with torch.no_grad():
        for j in (0, 37):
            h = abs(c0[j].item())
            fd = 0j
            for unit in (1.0, 1j):
                e = torch.zeros(64, dtype=c0.dtype, device="cuda")
                e[j] = unit * h
                d = (objective(c0 + e) - objective(c0 - e)).item() / (2 * h)
                fd += d * (1 if unit == 1.0 else 1j)
            print(f"coefficient {j}: autograd {g[j]:.6e}, central difference {fd:.6e}")
            assert abs(g[j] - fd) <= 1e-3 * np.max(np.abs(g))
