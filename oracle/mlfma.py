"""CPU MLFMA for the PIE operator (Section 3), FP64, stage by stage.

One MVM y = Z x is, in this order:
  a0  local coefficients: J|_t = a_t (r - c_t) + beta_t, sigma_t, and
      d_t = div J|_t + w^2 eps0 sigma_t = 2 a_t + w^2 eps0 sigma_t;
  a1  near field: exact pair moments (oracle.moments) over triangle pairs whose
      leaf boxes are neighbours (one-box buffer);
  a2  leaf aggregation: five radiated densities per leaf box (mu0 J as three
      components, sigma -- received by div f_m --, and d -- received by the
      pulses), S[b,c,p] = sum_t int_t rho_c(r') exp(-i kappa_L khat_p.(r'-C_b));
  a3  interpolation up the tree (levels L-1..3);
  a4  translation at every level 3..L with the diagonal operator of Eq. (5);
  a5  anterpolation down the tree;
  a6  leaf disaggregation with the conjugate (receiving) patterns;
  a7  assembly into RWG / pulse testing (Galerkin, Section 2).

Eq. (4) is used with kappa_l = k0 / s_l.  Reading for the scale factors (the
table of [jp045] is not reproduced in the paper): kappa_l a_l = x is the same at
every level that is small in wavelengths (s_l = k0 a_l / x), and s_l = 1 (the
standard diagonalization) once k0 a_l > x, with (tau, x, N_theta) chosen by the
error search in oracle/search_asd.py.  Reading for the inter-level transfer (the
paper is silent): patterns on the child's sphere of radius kappa_c are carried
to the parent's kappa_p by spherical-harmonic analysis to degree N_theta - 1,
multiplication of degree l by (kappa_p / kappa_c)^l (the small-argument
relation j_l(x) ~ s^l j_l(x/s) behind Eq. (5)), synthesis, and the phase shift
exp(-i kappa_p khat.(C_c - C_p)):  F = Y diag((kappa_p/kappa_c)^l) Y^H W.
Anterpolation is the transpose with conjugate phases (adjoint under the
quadrature weights).  Here Y uses scipy's spherical harmonics.

Pinned: tests/test_oracle_mlfma.py compares this operator with the dense
matrix of oracle.dense (relative error within the Eq. (4)-(5) accuracy), checks
that with x -> its near field alone it equals the dense product restricted to
near pairs exactly, and checks the filter against the Legendre addition
theorem.
"""
import numpy as np
from scipy.special import sph_harm_y

from . import constants as C
from .asd import alpha_tilde, angular_grid, far_offsets
from .mesh import build_topology, local_coefficients
from .moments import Geometry, pair_moments
from .quadrature import radon7
from .tree import build_tree


def interpolation_filter(khat, w, ntheta, ratio):
    """F[p, p'] = sum_{l < N_theta} ratio^l sum_m Y_lm(p) conj(Y_lm(p')) w_p'."""
    theta = np.arccos(np.clip(khat[:, 2], -1, 1))
    phi = np.arctan2(khat[:, 1], khat[:, 0])
    F = np.zeros((khat.shape[0], khat.shape[0]), np.complex128)
    for l in range(ntheta):
        for m in range(-l, l + 1):
            y = sph_harm_y(l, m, theta, phi)
            F += (ratio ** l) * np.outer(y, np.conj(y) * w)
    assert np.max(np.abs(F.imag)) < 1e-10
    return F.real


class MLFMA:
    def __init__(self, xyz, tri, k0, L, tau=7, x=0.08, ntheta=8, side=0.0):
        self.top = build_topology(xyz, tri)
        self.geo = Geometry(xyz, tri)
        self.k0 = float(k0)
        self.w = C.omega_of_k(k0)
        self.L = L
        self.tau, self.x, self.ntheta = tau, x, ntheta
        self.tree = tr = build_tree(self.top.centroid, self.top.xyz, L, side)
        # near-singular pairs (oracle.moments) must all be near at the leaves:
        # a centroid distance below 1.5 h is below the leaf size only if a >= 1.5 h
        if tr.box_size(L) * tr.box_size(L) < 2.25 * float(np.max(self.geo.h2)):
            raise ValueError("leaf box smaller than 1.5 x the longest triangle edge")
        self.khat, self.wq = angular_grid(ntheta)
        self.P = self.khat.shape[0]
        # s_l = min(k0 a_l / x, 1): scaled plane waves for boxes small in
        # wavelengths, the standard diagonalization (s = 1) for larger ones
        self.kappa = {l: max(x / tr.box_size(l), k0) for l in range(1, L + 1)}
        self.scale = {l: k0 / self.kappa[l] for l in range(1, L + 1)}
        self._tables()
        self._near()

    # ---------------------------------------------------------------- setup
    def _tables(self):
        tr, L, P = self.tree, self.L, self.P
        perm = tr.perm
        T = perm.size
        # leaf box of every tree-ordered triangle
        self.tri_box = np.repeat(np.arange(tr.keys[L].size), np.diff(tr.leaf_start))
        Cb = tr.box_centers(L)[self.tri_box]                       # [T,3]
        b7, w7 = radon7()
        q = self.geo.q7[perm]                                       # [T,7,3]
        wq = self.geo.w7[perm]
        ph = np.exp(-1j * self.kappa[L] * np.einsum("tqd,pd->tqp", q - Cb[:, None, :], self.khat))
        self.Pi = np.einsum("tq,tqp->tp", wq, ph)                   # [T,P]
        u = q - self.geo.cent[perm][:, None, :]
        self.M = np.einsum("tq,tqd,tqp->tdp", wq, u, ph)           # [T,3,P]
        offs = far_offsets()
        self.trans = {}
        for l in range(3, L + 1):
            a = tr.box_size(l)
            Tl = np.zeros((offs.shape[0], P), np.complex128)
            for i, d in enumerate(offs):
                Tl[i] = alpha_tilde(self.k0, self.scale[l], self.tau, d * a, self.khat)
            self.trans[l] = (1j * self.k0 / (16 * np.pi ** 2)) * self.wq[None, :] * Tl
        self.F = {}
        self.phase = {}
        for l in range(2, L):
            ratio = self.kappa[l] / self.kappa[l + 1]
            self.F[l] = interpolation_filter(self.khat, self.wq, self.ntheta, ratio)
            half = tr.box_size(l + 1) * 0.5
            ph = np.zeros((8, P), np.complex128)
            for o in range(8):
                dvec = half * np.array([2 * ((o >> 2) & 1) - 1, 2 * ((o >> 1) & 1) - 1, 2 * (o & 1) - 1])
                ph[o] = np.exp(-1j * self.kappa[l] * (self.khat @ dvec))
            self.phase[l] = ph

    def _near(self):
        tr, L = self.tree, self.L
        tt, ss = [], []
        for b in range(tr.keys[L].size):
            tests = np.arange(tr.leaf_start[b], tr.leaf_start[b + 1])
            srcs = np.concatenate([np.arange(tr.leaf_start[n], tr.leaf_start[n + 1])
                                   for n in tr.near_idx[tr.near_ptr[b]:tr.near_ptr[b + 1]]])
            for t in tests:
                tt.append(np.full(srcs.size, t))
                ss.append(srcs)
        self.near_t = np.concatenate(tt)      # tree-order indices
        self.near_s = np.concatenate(ss)
        perm = tr.perm
        self.near_m = pair_moments(self.geo, self.k0, perm[self.near_t], perm[self.near_s])

    # ---------------------------------------------------------------- apply
    def coefficients(self, x):
        a, beta, sig = local_coefficients(self.top, x)
        perm = self.tree.perm
        a, beta, sig = a[perm], beta[perm], sig[perm]
        d = 2.0 * a + self.w * self.w * C.EPS0 * sig
        return a, beta, sig, d

    def near_potentials(self, coef):
        a, beta, sig, d = coef
        m0, mt, ms, mts = self.near_m
        t, s = self.near_t, self.near_s
        T = a.size
        U = np.zeros(T, np.complex128)
        V = np.zeros((T, 3), np.complex128)
        T1 = np.zeros(T, np.complex128)
        T2 = np.zeros(T, np.complex128)
        np.add.at(U, t, C.MU0 * (a[s] * mts + np.sum(beta[s] * mt, axis=1)))
        np.add.at(V, t, C.MU0 * (a[s][:, None] * ms + beta[s] * m0[:, None]))
        np.add.at(T1, t, sig[s] * m0)
        np.add.at(T2, t, d[s] * m0)
        return U, V, T1, T2

    def aggregate(self, coef):
        a, beta, sig, d = coef
        contrib = np.zeros((a.size, 5, self.P), np.complex128)
        contrib[:, 0:3] = C.MU0 * (a[:, None, None] * self.M + beta[:, :, None] * self.Pi[:, None, :])
        contrib[:, 3] = sig[:, None] * self.Pi
        contrib[:, 4] = d[:, None] * self.Pi
        tr = self.tree
        return np.add.reduceat(contrib, tr.leaf_start[:-1], axis=0)

    def far_patterns(self, coef, levels=None):
        """Stage outputs: S[l] radiated patterns and G[l] incoming patterns.
        ``levels`` (optional) keeps the translations of those levels only."""
        tr, L = self.tree, self.L
        S = {L: self.aggregate(coef)}
        for l in range(L - 1, 2, -1):
            Sc = S[l + 1] @ self.F[l].T                          # [nc,5,P]
            octs = tr.keys[l + 1] & 7
            Sc = Sc * self.phase[l][octs][:, None, :]
            Sp = np.zeros((tr.keys[l].size, 5, self.P), np.complex128)
            np.add.at(Sp, tr.parent[l + 1], Sc)
            S[l] = Sp
        G = {}
        for l in range(3, L + 1):
            ptr, src, off = tr.il_ptr[l], tr.il_idx[l], tr.il_off[l]
            dst = np.repeat(np.arange(tr.keys[l].size), np.diff(ptr))
            Gl = np.zeros_like(S[l])
            if levels is None or l in levels:
                np.add.at(Gl, dst, self.trans[l][off][:, None, :] * S[l][src])
            G[l] = Gl
        for l in range(3, L):
            octs = tr.keys[l + 1] & 7
            H = G[l][tr.parent[l + 1]] * np.conj(self.phase[l][octs])[:, None, :]
            G[l + 1] = G[l + 1] + H @ self.F[l]
        return S, G

    def disaggregate(self, GL):
        g = GL[self.tri_box]                                     # [T,5,P]
        cPi = np.conj(self.Pi)
        cM = np.conj(self.M)
        U = np.einsum("tdp,tdp->t", cM, g[:, 0:3])
        V = np.einsum("tp,tdp->td", cPi, g[:, 0:3])
        T1 = np.einsum("tp,tp->t", cPi, g[:, 3])
        T2 = np.einsum("tp,tp->t", cPi, g[:, 4])
        return U, V, T1, T2

    def assemble(self, pots):
        """Galerkin testing of per-triangle potentials -> y (mesh order)."""
        U, V, T1, T2 = pots
        top, perm = self.top, self.tree.perm
        E = top.E
        y = np.zeros(top.N, np.complex128)
        for i, t in enumerate(perm):
            for k in range(3):
                n = top.tri_edges[t, k]
                if n < 0:
                    continue
                s = top.tri_sign[t, k]
                p = top.xyz[top.edge_free[n, 0 if s > 0 else 1]]
                c = s * top.edge_len[n] / (2.0 * top.area[t])
                y[n] += c * (U[i] + np.dot(top.centroid[t] - p, V[i])) + 2.0 * c * T1[i]
            y[E + t] += T2[i]
        return y

    def apply(self, x, near=True, far=True, stages=False, levels=None):
        """y = Z x; near / far switch the two parts, ``levels`` keeps the
        translations of those tree levels only (oracle.levels)."""
        coef = self.coefficients(x)
        T = coef[0].size
        pots = [np.zeros(T, np.complex128), np.zeros((T, 3), np.complex128),
                np.zeros(T, np.complex128), np.zeros(T, np.complex128)]
        S = G = None
        if near:
            pots = [p + q for p, q in zip(pots, self.near_potentials(coef))]
        if far:
            S, G = self.far_patterns(coef, levels)
            pots = [p + q for p, q in zip(pots, self.disaggregate(G[self.L]))]
        y = self.assemble(pots)
        if stages:
            return y, dict(coef=coef, S=S, G=G, pots=pots)
        return y
