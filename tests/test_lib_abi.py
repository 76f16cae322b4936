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


def test_problem_parameter_validation_on_host(libpie):
    """Invalid parameters and a too-small leaf box are rejected before any
    device work (these calls need no GPU)."""
    import paper_1806_04164_gb300 as pg
    xyz, tri = pi.icosphere(2)
    m = pg.Mesh(xyz, tri)
    bad = [dict(levels=2), dict(levels=3, tau=31), dict(levels=3, ntheta=7), dict(levels=3, kappa_a=0.0),
           dict(levels=3, precision=4), dict(levels=3, precision=-1), dict(levels=3, max_nrhs=0)]
    for kw in bad:
        with pytest.raises(pg.PieError) as ei:
            pg.Problem(m, 0.01, root_side=2.0, stream=0, **kw)
        assert ei.value.code == 1, kw
    with pytest.raises(pg.PieError) as ei:
        pg.Problem(m, -1.0, 3, root_side=2.0, stream=0)
    assert ei.value.code == 1
    with pytest.raises(pg.PieError) as ei:
        pg.Problem(m, 0.01, 4, root_side=2.0, stream=0)        # leaf 0.25 m < 1.5 x longest edge
    assert ei.value.code == 7
    with pytest.raises(pg.PieError) as ei:
        pg.Problem(m, 30.0, 3, root_side=2.0, stream=0)        # not a low-frequency problem
    assert ei.value.code == 1


def test_group_and_tuning_argument_checks_on_host(libpie):
    """Argument checks of the tuning and group calls need no GPU."""
    import ctypes
    import paper_1806_04164_gb300 as pg
    L = pg.lib()
    out = ctypes.c_void_p()
    assert L.pie_group_create(None, 1, ctypes.byref(out)) == 1
    arr = (ctypes.c_void_p * 1)(None)
    assert L.pie_group_create(arr, 1, ctypes.byref(out)) == 1
    assert L.pie_group_create(arr, 0, ctypes.byref(out)) == 1
    assert L.pie_group_apply(None, None, None, 1, None) == 1
    assert L.pie_group_info(None, None, None) == 1
    L.pie_group_destroy(None)
    t = pg.Tuning(1, 2, 1, 0)
    assert L.pie_problem_set_tuning(None, ctypes.byref(t)) == 1
    assert L.pie_problem_get_tuning(None, ctypes.byref(t)) == 1
    assert L.pie_problem_autotune(None, 1, 3, ctypes.byref(t), None, None) == 1
    xyz, tri = pi.icosphere(1)
    m = pg.Mesh(xyz, tri)
    p = pg.Params(3, 2.0, 7, 0.08, 8, 0, 1)
    best = ctypes.c_int32()
    assert L.pie_tune_levels(m.handle, 0.01, ctypes.byref(p), 2, 4, 1, None, ctypes.byref(best), None) == 1
    assert L.pie_tune_levels(m.handle, 0.01, ctypes.byref(p), 5, 4, 1, None, ctypes.byref(best), None) == 1
