"""Search for the Eq. (4)-(5) parameters (tau, x = kappa a, N_theta), in FP64
and in emulated FP32 (test infrastructure, like the rest of this package).

The paper tabulates optimal truncation numbers and scale factors per box size
(Section 3, citing [jp045]) but does not print the table.  This module
regenerates the choice: for one-box-buffer geometries (source and observation
boxes of side a at the 316 far offsets, points uniform in each box) it
evaluates Eq. (4) with Eq. (5) and reports the RMS and maximum relative error
against exact g.  At low frequency (k a << 1) the error depends on
x = (k/s) a, tau and N_theta only, so one triple serves every level.

Two evaluations of the same discretised Eq. (4):

* FP64: every step in double precision.
* emulated FP32: the translation operator is built in FP64 and rounded to
  complex float (its scaled Hankel terms s^t h_t(k w) overflow float for
  small k w), the point coordinates are rounded to float, the plane-wave
  phases exp(-/+ i kappa khat.(r - C)) are evaluated from them in float, and
  the angular sum runs in complex float, sample after sample.

Rounding amplification: the angular sum of Eq. (4) cancels terms far larger
than its result -- the degree-t term of Eq. (5) grows like (2t+1)!! / (kappa w)^t
-- so a relative rounding error eps of the summands becomes eps * cond in the
result, cond = sum_p |w_p alpha(khat_p) ...| / |g|.  ``amplification``
returns the largest cond over the sampled geometries.

Run:  python -m oracle.search_asd   (prints the table; a few minutes)
Pinned by tests/test_oracle_search_asd.py: FP32 and FP64 agree where the
amplification is small, the FP32 excess follows eps_32 * cond, and the
approximation error of the scaled plane waves grows as x^2 (the first
neglected term of j_t(z) ~ s^t j_t(z/s), Eq. (5)).
"""
import numpy as np

from .asd import alpha_tilde, angular_grid, far_offsets

EPS32 = float(np.finfo(np.float32).eps) / 2   # unit roundoff of float
EPS64 = float(np.finfo(np.float64).eps) / 2


def geometries(a, npair, npts, seed):
    """npair box pairs at random far offsets, npts random points in each box."""
    rng = np.random.default_rng(seed)
    offs = far_offsets()
    out = []
    for _ in range(npair):
        d = offs[rng.integers(len(offs))]
        Co, Cs = d * a, np.zeros(3)
        r = Co + (rng.random((npts, 3)) - 0.5) * a
        rp = Cs + (rng.random((npts, 3)) - 0.5) * a
        out.append((Co, Cs, r, rp))
    return out


def eq4_terms(k, s, tau, ntheta, r, rp, Co, Cs):
    """Summands of the discretised Eq. (4) for the point pairs (r, rp):
    prefactor * w_p * alpha(khat_p) and the two plane-wave phase factors, all
    in FP64 ([P], [M, P], [M, P])."""
    khat, w = angular_grid(ntheta)
    kap = k / s
    al = (1j * k / (16.0 * np.pi ** 2)) * w * alpha_tilde(k, s, tau, np.asarray(Co) - np.asarray(Cs), khat)
    ph_o = np.exp(1j * kap * ((r - Co) @ khat.T))
    ph_s = np.exp(-1j * kap * ((rp - Cs) @ khat.T))
    return al, ph_o, ph_s


def green_fp64(k, s, tau, ntheta, r, rp, Co, Cs):
    al, ph_o, ph_s = eq4_terms(k, s, tau, ntheta, r, rp, Co, Cs)
    return (ph_o * ph_s) @ al


def green_fp32(k, s, tau, ntheta, r, rp, Co, Cs):
    """Eq. (4) in emulated FP32 (see the module header); returns complex128
    holding the float result."""
    khat, w = angular_grid(ntheta)
    kap = np.float32(k / s)
    al = ((1j * k / (16.0 * np.pi ** 2)) * w * alpha_tilde(k, s, tau, np.asarray(Co) - np.asarray(Cs), khat))
    al32 = al.astype(np.complex64)
    kh32 = khat.astype(np.float32)
    dr = (r.astype(np.float32) - np.asarray(Co).astype(np.float32))
    ds = (rp.astype(np.float32) - np.asarray(Cs).astype(np.float32))
    arg_o = (kap * (dr @ kh32.T)).astype(np.float32)
    arg_s = (kap * (ds @ kh32.T)).astype(np.float32)
    ph_o = (np.cos(arg_o) + 1j * np.sin(arg_o)).astype(np.complex64)
    ph_s = (np.cos(arg_s) - 1j * np.sin(arg_s)).astype(np.complex64)
    terms = (ph_o * (ph_s * al32[None, :]).astype(np.complex64)).astype(np.complex64)
    # sequential float accumulation over the samples
    return np.cumsum(terms, axis=1, dtype=np.complex64)[:, -1].astype(np.complex128)


def exact_g(k, r, rp):
    R = np.linalg.norm(r - rp, axis=1)
    return np.exp(1j * k * R) / (4 * np.pi * R)


def pair_errors(k, a, x, tau, ntheta, npair=60, npts=30, seed=0, fp32=False):
    """(RMS, max) relative error of Eq. (4)-(5) against exact g."""
    s = k * a / x
    errs = []
    f = green_fp32 if fp32 else green_fp64
    for Co, Cs, r, rp in geometries(a, npair, npts, seed):
        g = exact_g(k, r, rp)
        errs.append(np.abs(f(k, s, tau, ntheta, r, rp, Co, Cs) - g) / np.abs(g))
    e = np.concatenate(errs)
    return float(np.sqrt(np.mean(e ** 2))), float(e.max())


def amplification(k, a, x, tau, ntheta, npair=60, npts=30, seed=0):
    """Largest ratio sum_p |summand_p| / |g| over the sampled point pairs: the
    factor by which a relative rounding error of the summands reaches g."""
    s = k * a / x
    worst = 0.0
    for Co, Cs, r, rp in geometries(a, npair, npts, seed):
        al, ph_o, ph_s = eq4_terms(k, s, tau, ntheta, r, rp, Co, Cs)
        mag = np.abs(ph_o * ph_s) @ np.abs(al)
        worst = max(worst, float(np.max(mag / np.abs(exact_g(k, r, rp)))))
    return worst


def scan(k=1e-3, a=0.0625, taus=range(2, 13), xs=(0.02, 0.03, 0.05, 0.08, 0.1, 0.15, 0.2, 0.3, 0.5, 1.0, 2.0),
         npair=40, npts=20):
    """Rows (tau, N_theta, P, x, rms64, max64, rms32, max32, cond) over the
    grid; N_theta from tau/2 + 2 up to tau + 4 (even values, at most 16)."""
    rows = []
    for tau in taus:
        nths = sorted({n + (n & 1) for n in (tau // 2 + 2, (3 * tau) // 4 + 3, tau + 4)})
        for nth in (n for n in nths if n <= 16):
            for x in xs:
                r64, m64 = pair_errors(k, a, x, tau, nth, npair, npts)
                r32, m32 = pair_errors(k, a, x, tau, nth, npair, npts, fp32=True)
                cond = amplification(k, a, x, tau, nth, npair, npts)
                rows.append(dict(tau=tau, ntheta=nth, P=2 * nth * nth, x=x, rms64=r64, max64=m64, rms32=r32,
                                 max32=m32, cond=cond))
    return rows


def choose(rows, rms_cap, max_cap, fp32, eps_cond_cap):
    """Cheapest point (fewest samples P, then lowest RMS) whose error in the
    given arithmetic stays within the caps and whose rounding term
    eps * cond stays below eps_cond_cap."""
    eps = EPS32 if fp32 else EPS64
    ok = [r for r in rows if (r["rms32"] if fp32 else r["rms64"]) <= rms_cap
          and (r["max32"] if fp32 else r["max64"]) <= max_cap and eps * r["cond"] <= eps_cond_cap]
    if not ok:
        return None
    return min(ok, key=lambda r: (r["P"], r["rms32"] if fp32 else r["rms64"]))


def main():
    rows = scan()
    print("tau N_th    P     x     rms64     max64     rms32     max32      cond")
    for r in rows:
        print(f"{r['tau']:3d} {r['ntheta']:4d} {r['P']:4d} {r['x']:5.2f} {r['rms64']:9.2e} {r['max64']:9.2e} "
              f"{r['rms32']:9.2e} {r['max32']:9.2e} {r['cond']:9.2e}")


if __name__ == "__main__":
    main()
