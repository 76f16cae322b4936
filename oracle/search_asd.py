"""Search for the Eq. (4)-(5) parameters (tau, x = kappa a, N_theta).

The paper tabulates optimal truncation numbers and scale factors per box size
(Section 3, citing [jp045]) but does not print the table.  This script
regenerates the choice: for one-box-buffer geometries (source and observation
boxes of side a at the 316 far offsets, points uniform in each box) it
evaluates Eq. (4) with Eq. (5) in FP64 and reports the RMS and maximum relative
error against exact g.  At low frequency (k a << 1) the error depends on
x = (k/s) a, tau and N_theta only, so one triple serves every level.

Run:  python -m oracle.search_asd   (prints a table; about a minute)
"""
import numpy as np

from .asd import far_offsets, green_asd


def pair_errors(k, a, x, tau, ntheta, npair=60, npts=30, seed=0):
    rng = np.random.default_rng(seed)
    offs = far_offsets()
    s = k * a / x
    errs = []
    for _ in range(npair):
        d = offs[rng.integers(len(offs))]
        Co, Cs = d * a, np.zeros(3)
        r = Co + (rng.random((npts, 3)) - 0.5) * a
        rp = Cs + (rng.random((npts, 3)) - 0.5) * a
        R = np.linalg.norm(r - rp, axis=1)
        g = np.exp(1j * k * R) / (4 * np.pi * R)
        errs.append(np.abs(green_asd(k, s, tau, ntheta, r, rp, Co, Cs) - g) / np.abs(g))
    e = np.concatenate(errs)
    return float(np.sqrt(np.mean(e ** 2))), float(e.max())


def main():
    print("k a        tau N_th  P    x      rms       max")
    for k, a in ((1e-2, 0.5), (1e-3, 0.0625), (1e-4, 2.0 / 256)):
        for tau, nth in ((4, 5), (5, 6), (6, 7), (7, 7), (7, 8), (8, 9)):
            best = None
            for x in (0.01, 0.015, 0.02, 0.03, 0.04, 0.05, 0.06, 0.07, 0.09):
                rms, mx = pair_errors(k, a, x, tau, nth)
                if best is None or rms < best[1]:
                    best = (x, rms, mx)
            print(f"{k * a:8.2e}  {tau:3d} {nth:4d} {2 * nth * nth:4d} {best[0]:6.3f} {best[1]:9.2e} {best[2]:9.2e}")


if __name__ == "__main__":
    main()
