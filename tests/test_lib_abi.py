"""CPU tests of the C ABI: the library builds, exports every function the
header declares, and its host-side mesh logic matches the oracle bit for bit.
No compute call is made (no GPU here)."""
import ctypes

import numpy as np
import pytest

import pie_inputs as pi
from oracle.mesh import build_topology
from tests._lib import ensure_built, header_functions


@pytest.fixture(scope="module")
def libpie():
    path = ensure_built()
    return ctypes.CDLL(path)


def test_exports_every_declared_function(libpie):
    import paper_1806_04164_gb300 as pg
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(libpie, n), n
    assert sorted(pg.EXPORTS) == names


@pytest.mark.parametrize("n", [0, 2, 3])
def test_mesh_edges_bit_exact(libpie, n):
    import paper_1806_04164_gb300 as pg
    xyz, tri = pi.icosphere(n)
    m = pg.Mesh(xyz, tri)
    top = build_topology(xyz, tri)
    e, et, ef = m.edges()
    assert m.ne == top.E and m.nt == top.T
    assert np.array_equal(e, top.edges)
    assert np.array_equal(et, top.edge_tri)
    assert np.array_equal(ef, top.edge_free)


def test_open_surface_and_errors(libpie):
    import paper_1806_04164_gb300 as pg
    xyz, tri = pi.flat_pair("edge")
    m = pg.Mesh(xyz, tri)
    assert m.ne == 1 and m.nt == 2
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, -1, 0.5]], float)
    with pytest.raises(pg.PieError) as ei:
        pg.Mesh(xyz, np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]]))
    assert ei.value.code == 2
    with pytest.raises(pg.PieError) as ei:
        pg.Mesh(np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0.]]), np.array([[0, 1, 2]]))
    assert ei.value.code == 3
    with pytest.raises(pg.PieError) as ei:
        pg.Mesh(xyz, np.array([[0, 1, 2], [0, 1, 3]]))
    assert ei.value.code == 4
    with pytest.raises(pg.PieError) as ei:
        pg.Mesh(xyz, np.array([[0, 1, 7]]))
    assert ei.value.code == 1
