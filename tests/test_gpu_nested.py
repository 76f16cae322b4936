"""The complex-float inner operator and the nested solve (Section 4 solves
with GMRES; the far part is the same Eqs. (4)-(5) operator at a point whose
rounding amplification complex float tolerates).

* PIE_FP32H: near pair moments stored as half precision with a power-of-two
  scale per moment plane.  Every stored moment must equal the FP64 moment to
  half's unit roundoff (2^-11 relative) plus float rounding of the plane's
  largest entry; products equal the PIE_FP32 ones to that rounding.
* pie_solve_nested: flexible GMRES on the FP64-far operator with inner
  GMRES cycles on a complex-float operator.  Its solution must satisfy the
  outer system to the requested tolerance (checked with an independent
  product), give the same far field as pie_solve and the Mie series, and
  agree with the dense oracle solution as closely as pie_solve's does.
"""
import numpy as np
import pytest

import pie_inputs as pi

pytestmark = pytest.mark.gpu
K = 0.01
INNER = dict(tau=3, kappa_a=0.15, ntheta=4)   # the nested solver's inner Eq. (4)-(5) point


@pytest.fixture(scope="module")
def pg():
    from tests._lib import ensure_built
    ensure_built()
    import paper_1806_04164_gb300 as pg
    return pg


@pytest.fixture(scope="module")
def mesh3():
    return pi.icosphere(3)


def rel(a, b):
    import torch
    a = a.cpu().numpy() if torch.is_tensor(a) else a
    b = b.cpu().numpy() if torch.is_tensor(b) else b
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_half_moments_round_the_fp64_moments(pg, mesh3):
    p64 = pg.Problem(pg.Mesh(*mesh3), K, 4, root_side=2.0, **INNER)
    p16 = pg.Problem(pg.Mesh(*mesh3), K, 4, root_side=2.0, precision=pg.PIE_FP32H, **INNER)
    m64, m16 = p64.stage(4), p16.stage(4)
    for q in range(8):
        top = np.max(np.abs(m64[q]))
        # real and imaginary parts are rounded separately
        err = np.maximum(np.abs(m16[q].real - m64[q].real), np.abs(m16[q].imag - m64[q].imag))
        bound = 2.0 ** -11 * np.maximum(np.abs(m64[q].real), np.abs(m64[q].imag)) + 2.0 ** -23 * top
        assert np.all(err <= bound), q
    # half the near-part bytes of PIE_FP32
    p32 = pg.Problem(pg.Mesh(*mesh3), K, 4, root_side=2.0, precision=pg.PIE_FP32, **INNER)
    assert p32.device_bytes - p16.device_bytes == 4 * 8 * p16.near_pairs


def test_half_moment_products(pg, mesh3):
    import torch
    p64 = pg.Problem(pg.Mesh(*mesh3), K, 4, root_side=2.0, **INNER)
    p32 = pg.Problem(pg.Mesh(*mesh3), K, 4, root_side=2.0, precision=pg.PIE_FP32, **INNER)
    p16 = pg.Problem(pg.Mesh(*mesh3), K, 4, root_side=2.0, precision=pg.PIE_FP32H, **INNER)
    x = torch.from_numpy(pi.complex_normal(p64.N, 11)).cuda()
    xf = x.to(torch.complex64)
    yn = p64.apply(x, near_only=True)
    assert rel(p16.apply(xf, near_only=True).to(torch.complex128), yn) < 1e-3
    assert rel(p32.apply(xf, near_only=True).to(torch.complex128), yn) < 1e-5
    # the far part runs the same float kernels: the products differ by the moments' rounding
    y32, y16 = p32.apply(xf), p16.apply(xf)
    assert rel(y16, y32) < 1e-3
    # at this low-amplification point float keeps the product close to FP64
    assert rel(y32.to(torch.complex128), p64.apply(x)) < 1e-4
    # the allocation-free near product reads the half moments too
    yna = torch.empty_like(xf)
    pg.lib().pie_apply_near_noalloc(p16.handle, pg.ctypes.c_void_p(xf.data_ptr()), pg.ctypes.c_void_p(yna.data_ptr()),
                                    pg.PIE_C64, pg._stream(None))
    assert torch.equal(yna, p16.apply(xf, near_only=True))


def test_small_grid_fp64_matches_oracle(pg, mesh3):
    """N_theta = 4 (P = 32) packs several boxes per block in the aggregation
    and translation kernels: stages and product against the oracle MLFMA at
    the inner operator's point (amplification ~1e3: rounding-level agreement)."""
    import torch
    from oracle.mlfma import MLFMA
    L = 4
    M = MLFMA(*mesh3, K, L, tau=INNER["tau"], x=INNER["kappa_a"], ntheta=INNER["ntheta"], side=2.0)
    pr = pg.Problem(pg.Mesh(*mesh3), K, L, root_side=2.0, **INNER)
    x = pi.complex_normal(pr.N, 1234)
    y = pr.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    yo, st = M.apply(x, stages=True)
    for l in range(3, L + 1):
        S, G = pr.stage(0, l), pr.stage(1, l)
        for c in range(5):
            assert rel(S[:, c], st["S"][l][:, c]) < 1e-12, ("S", l, c)
            assert rel(G[:, c], st["G"][l][:, c]) < 1e-12, ("G", l, c)
    assert rel(y, yo) < 1e-11


@pytest.fixture(scope="module")
def pair(pg, mesh3):
    mesh = pg.Mesh(*mesh3)
    outer = pg.Problem(mesh, K, 4, root_side=2.0, precision=pg.PIE_MIXED)
    inner = pg.Problem(mesh, K, 4, root_side=2.0, precision=pg.PIE_FP32H, **INNER)
    return outer, inner


@pytest.mark.parametrize("outer_restart", [20, 0])
def test_nested_solution_satisfies_outer_system(pg, pair, outer_restart):
    """Flexible GMRES (outer_restart 20) and iterative refinement
    (outer_restart 0): the residual with the outer operator, recomputed by
    an independent product, meets the tolerance (up to the outer operator's
    ~3e-6 rounding nonlinearity), and the far field equals that of pie_solve."""
    import torch
    from oracle import mie
    outer, inner = pair
    b = outer.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    x, st = outer.solve_nested(b, inner, tol=1e-6, maxit=6000, inner_restart=20, inner_tol=0.1,
                               outer_restart=outer_restart, max_outer=400)
    assert st["converged"] and st["rel_residual"] <= 1e-6, st
    assert st["inner_iterations"] > 0 and st["outer_products"] >= 1
    r = b - outer.apply(x)
    assert torch.linalg.norm(r).item() <= 5e-6 * torch.linalg.norm(b).item()
    xr, sr = outer.solve(b, tol=1e-6, maxit=3000, restart=100)
    rh = pi.bistatic_directions(181)
    E, Er = outer.farfield(x, rh).cpu().numpy(), outer.farfield(xr, rh).cpu().numpy()
    assert np.linalg.norm(E - Er) <= 1e-4 * np.linalg.norm(Er)
    s = 4 * np.pi * np.sum(np.abs(E) ** 2, axis=1)
    sm = mie.rcs_eplane(K, 1.0, -rh[:, 2])
    mask = sm > 1e-2 * sm.max()
    assert np.max(np.abs(10 * np.log10(s[mask] / sm[mask]))) < 0.1
    print("nested", st, "plain iterations", sr["iterations"])


def test_nested_matches_dense_solution(pg):
    """Against the oracle's dense solve on the 320-triangle sphere: the
    nested solution inherits the product's far-part accuracy (~1e-3), as
    pie_solve's does."""
    import torch
    from oracle.dense import assemble
    from oracle.excitation import rhs_planewave
    from oracle.mesh import build_topology
    xyz, tri = pi.icosphere(2)
    top = build_topology(xyz, tri)
    Z = assemble(top, K)
    bo = rhs_planewave(top, K, [0, 0, -1.0], [1.0, 0, 0])
    xo = np.linalg.solve(Z, bo)
    mesh = pg.Mesh(xyz, tri)
    outer = pg.Problem(mesh, K, 3, root_side=2.0)
    inner = pg.Problem(mesh, K, 3, root_side=2.0, precision=pg.PIE_FP32H, **INNER)
    x, st = outer.solve_nested(torch.from_numpy(bo).cuda(), inner, tol=1e-5, maxit=4000, inner_restart=20,
                               inner_tol=0.1, outer_restart=40, max_outer=200)
    assert st["converged"]
    x = x.cpu().numpy()
    E = top.E
    assert np.linalg.norm(x[:E] - xo[:E]) <= 1e-2 * np.linalg.norm(xo[:E])


def test_nested_argument_checks_and_zero_rhs(pg, pair, mesh3):
    import torch
    outer, inner = pair
    b = outer.rhs_planewave([0, 0, -1.0], [1.0, 0, 0])
    # inner problem on another mesh
    other = pg.Problem(pg.Mesh(*pi.icosphere(2)), K, 3, root_side=2.0, precision=pg.PIE_FP32)
    with pytest.raises(pg.PieError) as ei:
        outer.solve_nested(b, other)
    assert ei.value.code == 1
    # another wavenumber
    other = pg.Problem(pg.Mesh(*mesh3), 2 * K, 4, root_side=2.0, precision=pg.PIE_FP32H, **INNER)
    with pytest.raises(pg.PieError):
        outer.solve_nested(b, other)
    # complex-float outer problem, out-of-range parameters
    with pytest.raises(pg.PieError):
        inner.solve_nested(b.to(torch.complex64), inner)
    for kw in (dict(inner_tol=1.0), dict(inner_restart=0), dict(outer_restart=-1), dict(max_outer=0)):
        with pytest.raises(pg.PieError):
            outer.solve_nested(b, inner, **kw)
    # b = 0: x = 0 at once
    x, st = outer.solve_nested(torch.zeros_like(b), inner)
    assert st["converged"] and st["inner_iterations"] == 0 and torch.count_nonzero(x).item() == 0
    # an iteration budget too small reports non-convergence, not an error
    x, st = outer.solve_nested(b, inner, maxit=3, inner_restart=3, outer_restart=1, max_outer=2)
    assert not st["converged"] and st["inner_iterations"] <= 3


def test_solve_guess_with_zero_rhs_returns_zero(pg, pair):
    """pie_solve_guess with b = 0 and a nonzero initial guess: the solution
    of Z x = 0 is x = 0, whatever the guess."""
    import torch
    outer, _ = pair
    b = torch.zeros(outer.N, dtype=torch.complex128, device="cuda")
    x0 = torch.from_numpy(pi.complex_normal(outer.N, 3)).cuda()
    x, st = outer.solve(b, x0=x0)
    assert st["converged"] and torch.count_nonzero(x).item() == 0
