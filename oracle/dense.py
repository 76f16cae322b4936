"""Dense Galerkin matrix of the PIEs, Eqs. (1)-(2) (the O(N^2) MOM of Section 3).

Testing Eq. (1) with the RWG functions (tangential reading: <f_m, X> for the
equation n x X = -n x A^inc) and Eq. (2) with the pulses, and moving the
gradient of g onto the testing function by parts (Section 3: for RWG f_m,
<f_m, int sigma grad'g> = <div f_m, int sigma g>), gives the N x N system
(N = E + T, unknowns [x_J ; x_sigma] in mesh order):

  Z_JJ[m,n] = mu0      <f_m, g, f_n>
  Z_Js[m,t] =          <div f_m, g, p_t>
  Z_sJ[t,n] =          <p_t, g, div' f_n>
  Z_ss[t,u] = w^2 eps0 <p_t, g, p_u>

with <a, g, b> = int int a(r) . b(r') g(r, r') dr' dr.  Each entry is a sum of
the per-pair moments of oracle.moments over the triangles of the two basis
functions.  Pinned in tests/test_oracle_dense.py (complex symmetry, agreement
with an independent brute-force assembly from basis-function values on tiny
meshes, the static limit k -> 0).
"""
import numpy as np

from . import constants as C
from .mesh import Topology
from .moments import Geometry, pair_moments


def _rwg_tables(top: Topology):
    """Per triangle and local edge: RWG index, c = s l / (2A), div = s l / A,
    and (c_t - p) with p the free vertex."""
    T = top.T
    idx = top.tri_edges
    sgn = top.tri_sign.astype(np.float64)
    coef = np.zeros((T, 3))
    div = np.zeros((T, 3))
    dcp = np.zeros((T, 3, 3))
    for t in range(T):
        for k in range(3):
            n = idx[t, k]
            if n < 0:
                continue
            side = 0 if sgn[t, k] > 0 else 1
            p = top.xyz[top.edge_free[n, side]]
            coef[t, k] = sgn[t, k] * top.edge_len[n] / (2.0 * top.area[t])
            div[t, k] = sgn[t, k] * top.edge_len[n] / top.area[t]
            dcp[t, k] = top.centroid[t] - p
    return idx, coef, div, dcp


def assemble(top: Topology, k0: float, chunk=200000, pair_mask=None):
    """Dense N x N complex128 matrix Z (mesh order).

    ``pair_mask(t, s)`` (optional) keeps only the triangle pairs for which it
    returns True, e.g. to form the near-field part of Z alone."""
    E, T, N = top.E, top.T, top.N
    w = C.omega_of_k(k0)
    geo = Geometry(top.xyz, top.tri)
    idx, coef, div, dcp = _rwg_tables(top)
    Z = np.zeros((N, N), np.complex128)
    tt, ss = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    tt = tt.ravel()
    ss = ss.ravel()
    for a in range(0, tt.size, chunk):
        t = tt[a:a + chunk]
        s = ss[a:a + chunk]
        if pair_mask is not None:
            keep = pair_mask(t, s)
            t, s = t[keep], s[keep]
        m0, mt, ms, mts = pair_moments(geo, k0, t, s)
        # pulse-pulse
        np.add.at(Z, (E + t, E + s), w * w * C.EPS0 * m0)
        for kt in range(3):
            nt = idx[t, kt]
            okt = nt >= 0
            # RWG test, pulse source
            np.add.at(Z, (nt[okt], E + s[okt]), div[t[okt], kt] * m0[okt])
            for ks in range(3):
                ns = idx[s, ks]
                ok = okt & (ns >= 0)
                dt = dcp[t[ok], kt]
                ds = dcp[s[ok], ks]
                val = (mts[ok] + np.einsum("pd,pd->p", dt, ms[ok])
                       + np.einsum("pd,pd->p", mt[ok], ds)
                       + np.einsum("pd,pd->p", dt, ds) * m0[ok])
                np.add.at(Z, (nt[ok], ns[ok]), C.MU0 * coef[t[ok], kt] * coef[s[ok], ks] * val)
        for ks in range(3):
            ns = idx[s, ks]
            ok = ns >= 0
            np.add.at(Z, (E + t[ok], ns[ok]), div[s[ok], ks] * m0[ok])
    return Z


def rows(top: Topology, k0: float, which, x, pair_mask=None, sources=None):
    """Selected entries of y = Z x computed row by row without storing Z.

    ``which`` holds indices into the mesh-order unknown vector.  Used to check
    sampled outputs of large problems one by one.  ``pair_mask(t, s)`` keeps
    only the source triangles s (array) paired with test triangle t for which
    it returns True (e.g. the near part alone).  ``sources`` (optional) limits
    the sum to those source triangles (mesh order): the rows' partial sums
    over them.
    """
    E, T = top.E, top.T
    w = C.omega_of_k(k0)
    # geometry and RWG tables depend on the mesh only: built once per mesh
    cache = top.__dict__.setdefault("_rows_cache", {})
    if "geo" not in cache:
        cache["geo"] = Geometry(top.xyz, top.tri)
        cache["tables"] = _rwg_tables(top)
    geo = cache["geo"]
    tidx, tcoef, tdiv, tdcp = cache["tables"]
    x = np.asarray(x, np.complex128)
    xJ, xs = x[:E], x[E:]
    out = []
    allsrc = np.arange(T) if sources is None else np.asarray(sources, np.int64)
    idx, coef, div, dcp = tidx[allsrc], tcoef[allsrc], tdiv[allsrc], tdcp[allsrc]
    xs_src = xs[allsrc]
    for m in which:
        if m >= E:
            tests = [(m - E, None)]
        else:
            tests = [(int(top.edge_tri[m, 0]), m), (int(top.edge_tri[m, 1]), m)]
        acc = 0j
        for t, n in tests:
            tarr = np.full(allsrc.size, t)
            m0, mt, ms, mts = pair_moments(geo, k0, tarr, allsrc)
            if pair_mask is not None:
                keep = pair_mask(t, allsrc)
                m0, mt, ms, mts = m0 * keep, mt * keep[:, None], ms * keep[:, None], mts * keep
            if n is None:   # pulse test
                acc += np.sum(w * w * C.EPS0 * m0 * xs_src)
                for ks in range(3):
                    ns = idx[:, ks]
                    ok = ns >= 0
                    acc += np.sum(div[ok, ks] * m0[ok] * xJ[ns[ok]])
            else:           # RWG test
                kt = int(np.nonzero(tidx[t] == n)[0][0])
                acc += np.sum(tdiv[t, kt] * m0 * xs_src)
                dt = tdcp[t, kt]
                for ks in range(3):
                    ns = idx[:, ks]
                    ok = ns >= 0
                    ds = dcp[ok, ks]
                    val = (mts[ok] + ms[ok] @ dt + np.einsum("pd,pd->p", mt[ok], ds)
                           + (ds @ dt) * m0[ok])
                    acc += np.sum(C.MU0 * tcoef[t, kt] * coef[ok, ks] * val * xJ[ns[ok]])
        out.append(acc)
    return np.array(out)
