"""The stored Eq. (4)-(5) parameter search (tests/golden/asd_search.json,
written by tests/golden/make_asd_search.py from oracle/search_asd.py alone):
its rows are reproducible from the oracle, and the library's parameter points
are among the search's candidates -- the FP64 point of the accurate product
(chosen finally by its product-level error and rounding nonlinearity, which
pair-level errors do not capture) and the complex-float point of the nested
solver's inner operator (the search's first FP32 candidate)."""
import json
import os

import pytest

from oracle.search_asd import amplification, pair_errors

HERE = os.path.dirname(os.path.abspath(__file__))
K, A = 1e-3, 0.0625


@pytest.fixture(scope="module")
def table():
    with open(os.path.join(HERE, "golden", "asd_search.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("tau,ntheta,x", [(3, 4, 0.15), (7, 8, 0.08), (5, 6, 0.1)])
def test_rows_reproduce(table, tau, ntheta, x):
    row = next(r for r in table["rows"] if (r["tau"], r["ntheta"], r["x"]) == (tau, ntheta, x))
    r64, m64 = pair_errors(K, A, x, tau, ntheta, npair=40, npts=20)
    r32, m32 = pair_errors(K, A, x, tau, ntheta, npair=40, npts=20, fp32=True)
    cond = amplification(K, A, x, tau, ntheta, npair=40, npts=20)
    for got, want in ((r64, row["rms64"]), (m64, row["max64"]), (r32, row["rms32"]), (m32, row["max32"]),
                      (cond, row["cond"])):
        assert abs(got - want) <= 1e-9 * abs(want)   # reproducible up to the BLAS summation order


def test_library_points_are_candidates(table):
    import paper_1806_04164_gb300 as pg
    fp64 = [(r["tau"], r["ntheta"], r["x"]) for r in table["fp64_candidates"]]
    assert (pg.DEFAULT_TAU, pg.DEFAULT_NTHETA, pg.DEFAULT_KAPPA_A) in fp64
    first32 = table["fp32_candidates"][0]
    assert (first32["tau"], first32["ntheta"], first32["x"]) == (3, 4, 0.15)
    assert first32["rms32"] < 5e-3 and first32["P"] == 32
