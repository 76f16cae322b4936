"""Pins for the synthetic meshes (pie_inputs): counts, closedness, outward
orientation and enclosed volume against the closed forms."""
import numpy as np
import pytest

import pie_inputs as pi
from oracle.mesh import build_topology


def volume(xyz, tri):
    v0, v1, v2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    return np.sum(np.einsum("ij,ij->i", v0, np.cross(v1, v2))) / 6.0


@pytest.mark.parametrize("name,mesh,T,vol,tol", [
    ("sphere", lambda: pi.icosphere(3), 1280, 4 / 3 * np.pi, 1e-2),
    ("cube", lambda: pi.cube(32), 24576, 1.0, 1e-12),
    ("ellipsoid", lambda: pi.octasphere(6, (1.0, 0.5, 0.5)), 32768, 4 / 3 * np.pi * 0.25, 1e-3),
    ("cylinder", lambda: pi.cylinder(), 40960, np.pi * 0.25 * 2.0, 1e-3),
])
def test_closed_meshes(name, mesh, T, vol, tol):
    xyz, tri = mesh()
    top = build_topology(xyz, tri)
    assert top.T == T and top.E == 3 * T // 2
    assert xyz.shape[0] - top.E + top.T == 2
    v = volume(xyz, tri)
    assert v > 0 and abs(v - vol) <= tol * vol


def test_patch_is_open():
    xyz, tri = pi.square_patch(75)
    top = build_topology(xyz, tri)
    assert top.T == 11250 and top.E == 3 * 75 * 75 - 2 * 75
    assert np.all(top.normal[:, 2] > 0.999)


def test_planewave_set():
    """64 waves: 32 distinct unit directions, two unit polarisations each,
    both orthogonal to the direction and to each other."""
    w = pi.planewave_set()
    assert len(w) == 64
    dirs = {tuple(np.round(k, 12)) for k, _ in w}
    assert len(dirs) == 32
    for i in range(0, 64, 2):
        (k, e1), (k2, e2) = w[i], w[i + 1]
        assert np.allclose(k, k2)
        for v in (k, e1, e2):
            assert abs(np.linalg.norm(v) - 1) < 1e-14
        assert abs(k @ e1) < 1e-14 and abs(k @ e2) < 1e-14 and abs(e1 @ e2) < 1e-14
