"""Writes tests/golden/asd_search.json: the Eq. (4)-(5) parameter search of
oracle/search_asd.py (FP64 and emulated FP32 errors and the rounding
amplification over tau, N_theta and x = kappa a at k a = 6.25e-5), and the two
points chosen from it: the FP64 point of the accurate product and the FP32
point of the nested solver's inner operator.  Calls only the oracle.

Run:  python tests/golden/make_asd_search.py   (about a minute)
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.search_asd import EPS32, EPS64, scan  # noqa: E402


def main():
    rows = scan()
    # FP64 point: RMS <= 1e-3, max <= 5e-3, rounding term eps64 * cond <= 1e-4,
    # then the lowest amplification (GMRES reaches 1e-6 only below ~1e-5 of
    # rounding nonlinearity) among the points with the fewest samples
    fp64 = [r for r in rows if r["rms64"] <= 1e-3 and r["max64"] <= 5e-3 and EPS64 * r["cond"] <= 1e-4]
    # FP32 point: RMS <= 5e-3 in emulated FP32 and eps32 * cond <= 1e-3 (the
    # inner solver needs a low rounding nonlinearity more than accuracy),
    # fewest samples, then the lowest amplification
    fp32 = [r for r in rows if r["rms32"] <= 5e-3 and EPS32 * r["cond"] <= 1e-3]
    out = {"source": "oracle/search_asd.py scan(): one-box-buffer point pairs, k a = 6.25e-5",
           "rows": rows,
           "fp64_candidates": sorted(fp64, key=lambda r: (r["P"], -r["x"]))[:6],
           "fp32_candidates": sorted(fp32, key=lambda r: (r["P"], r["cond"]))[:6]}
    with open(os.path.join(HERE, "asd_search.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(len(rows), "rows;", "fp64:", [(r["tau"], r["ntheta"], r["x"]) for r in out["fp64_candidates"]],
          "fp32:", [(r["tau"], r["ntheta"], r["x"]) for r in out["fp32_candidates"]])


if __name__ == "__main__":
    main()
