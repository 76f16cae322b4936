"""Pins for oracle.asd (Eqs. (4)-(5))."""
import numpy as np

from oracle.asd import alpha_tilde, angular_grid, far_offsets, green_asd


def exact(k, r, rp):
    R = np.linalg.norm(r - rp, axis=1)
    return np.exp(1j * k * R) / (4 * np.pi * R)


def pts(rng, C, a, n=20):
    return C + (rng.random((n, 3)) - 0.5) * a


def test_grid_integrates_harmonics_exactly():
    for nt in (4, 8):
        khat, w = angular_grid(nt)
        assert abs(w.sum() - 4 * np.pi) < 1e-13
        # int x^a y^b z^c over the sphere, degree <= 2 nt - 1, against closed forms
        assert abs(np.sum(w * khat[:, 2] ** 2) - 4 * np.pi / 3) < 1e-13
        assert abs(np.sum(w * khat[:, 0] ** 2 * khat[:, 1] ** 2) - 4 * np.pi / 15) < 1e-13
        assert abs(np.sum(w * khat[:, 0] * khat[:, 1] * khat[:, 2])) < 1e-14


def test_s_equal_one_reduces_to_exact_diagonalization():
    """s = 1, large tau: Eq. (4) with the i k/(16 pi^2) prefactor reproduces g."""
    rng = np.random.default_rng(0)
    k, a = 8.0, 1.0
    Co = np.array([3.0, 2.0, 1.0]) * a
    Cs = np.zeros(3)
    r, rp = pts(rng, Co, a), pts(rng, Cs, a)
    ga = green_asd(k, 1.0, 40, 45, r, rp, Co, Cs)
    assert np.max(np.abs(ga - exact(k, r, rp)) / np.abs(exact(k, r, rp))) < 1e-10


def test_low_frequency_accuracy_of_chosen_parameters():
    """tau = 7, N_theta = 8, kappa a = 0.08 over one-box-buffer geometries at
    k a = 6e-5 and 5e-3: RMS relative error below 1e-3."""
    rng = np.random.default_rng(1)
    offs = far_offsets()
    for k, a in ((1e-3, 0.0625), (1e-2, 0.5)):
        s = k * a / 0.08
        errs = []
        for i in range(40):
            d = offs[rng.integers(len(offs))]
            Co, Cs = d * a, np.zeros(3)
            r, rp = pts(rng, Co, a), pts(rng, Cs, a)
            g = exact(k, r, rp)
            errs.append(np.abs(green_asd(k, s, 7, 8, r, rp, Co, Cs) - g) / np.abs(g))
        assert np.sqrt(np.mean(np.concatenate(errs) ** 2)) < 1e-3


def test_error_decreases_with_tau_until_rounding():
    rng = np.random.default_rng(2)
    k, a = 1e-3, 0.0625
    Co, Cs = np.array([2.0, 1.0, 0.0]) * a, np.zeros(3)
    r, rp = pts(rng, Co, a), pts(rng, Cs, a)
    g = exact(k, r, rp)
    e = [np.sqrt(np.mean(np.abs(green_asd(k, k * a / 0.06, t, 8, r, rp, Co, Cs) - g) ** 2 / np.abs(g) ** 2))
         for t in (1, 2, 3, 4, 5)]
    assert all(e[i + 1] < e[i] for i in range(4))


def test_offsets_and_symmetry():
    offs = far_offsets()
    assert offs.shape == (316, 3)
    assert len({tuple(o) for o in offs}) == 316
    khat, _ = angular_grid(6)
    a1 = alpha_tilde(1e-3, 1e-3, 5, np.array([0.2, 0.0, 0.1]), khat)
    a2 = alpha_tilde(1e-3, 1e-3, 5, -np.array([0.2, 0.0, 0.1]), -khat)
    assert np.allclose(a1, a2, rtol=1e-13)
