"""RWG / pulse discretisation of the PIE unknowns (Section 2, final paragraph).

J is expanded in RWG functions on the E interior edges, n'.A in pulse
functions on the T triangles; the unknown vector is ordered
[E RWG coefficients ; T pulse coefficients], N = T + E.

Readings (the paper is silent on these details):
* an interior edge is shared by exactly two triangles; edges are numbered in
  increasing (min vertex, max vertex) order;
* the "+" triangle of an edge is the one in whose counter-clockwise vertex
  order the edge runs from its smaller to its larger vertex index;
* f_n(r) = +(l_n / 2A+)(r - p+) on T+, -(l_n / 2A-)(r - p-) on T-, with p the
  vertex opposite the edge; div f_n = +-l_n / A+-;
* the pulse on triangle t is 1 on t and 0 elsewhere.

Pinned in tests/test_oracle_mesh.py (icosphere counts, Euler characteristic,
the RWG identity  int f_n dS = - int r div f_n dS  that fixes the sign of f
against its divergence, and the current-continuity of f_n across its edge).
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class Topology:
    xyz: np.ndarray          # [V,3]
    tri: np.ndarray          # [T,3]
    edges: np.ndarray        # [E,2] (vmin, vmax)
    edge_tri: np.ndarray     # [E,2] (T+, T-)
    edge_free: np.ndarray    # [E,2] free vertex in T+, T-
    edge_len: np.ndarray     # [E]
    area: np.ndarray         # [T]
    normal: np.ndarray       # [T,3] unit normal (ccw)
    centroid: np.ndarray     # [T,3]
    tri_edges: np.ndarray    # [T,3] RWG index of each local edge (or -1)
    tri_sign: np.ndarray     # [T,3] +1 / -1 / 0

    @property
    def T(self):
        return self.tri.shape[0]

    @property
    def E(self):
        return self.edges.shape[0]

    @property
    def N(self):
        return self.T + self.E


def build_topology(xyz, tri) -> Topology:
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    T = tri.shape[0]
    v0, v1, v2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    cr = np.cross(v1 - v0, v2 - v0)
    dbl = np.linalg.norm(cr, axis=1)
    if np.any(dbl <= 0):
        raise ValueError("degenerate triangle")
    area = 0.5 * dbl
    normal = cr / dbl[:, None]
    centroid = (v0 + v1 + v2) / 3.0

    # every (triangle, local edge) occurrence
    occ = {}
    for t in range(T):
        for k in range(3):
            a, b = int(tri[t, k]), int(tri[t, (k + 1) % 3])
            free = int(tri[t, (k + 2) % 3])
            key = (min(a, b), max(a, b))
            sign = 1 if a < b else -1
            occ.setdefault(key, []).append((t, k, sign, free))
    interior = sorted(k for k, v in occ.items() if len(v) == 2)
    for k, v in occ.items():
        if len(v) > 2:
            raise ValueError("non-manifold edge")
    E = len(interior)
    edges = np.array(interior, dtype=np.int64).reshape(E, 2)
    edge_tri = np.zeros((E, 2), np.int64)
    edge_free = np.zeros((E, 2), np.int64)
    tri_edges = -np.ones((T, 3), np.int64)
    tri_sign = np.zeros((T, 3), np.int64)
    for n, key in enumerate(interior):
        (ta, ka, sa, fa), (tb, kb, sb, fb) = occ[key]
        if sa == sb:
            raise ValueError("inconsistent orientation")
        if sa < 0:
            (ta, ka, sa, fa), (tb, kb, sb, fb) = (tb, kb, sb, fb), (ta, ka, sa, fa)
        edge_tri[n] = (ta, tb)
        edge_free[n] = (fa, fb)
        tri_edges[ta, ka], tri_sign[ta, ka] = n, 1
        tri_edges[tb, kb], tri_sign[tb, kb] = n, -1
    edge_len = np.linalg.norm(xyz[edges[:, 0]] - xyz[edges[:, 1]], axis=1)
    return Topology(xyz, tri, edges, edge_tri, edge_free, edge_len, area, normal,
                    centroid, tri_edges, tri_sign)


def rwg_values(top: Topology, n: int, t: int, r):
    """Value of RWG function n at points r [...,3] of triangle t (zero if t is
    not one of its triangles)."""
    r = np.asarray(r, dtype=np.float64)
    for side, s in ((0, 1.0), (1, -1.0)):
        if top.edge_tri[n, side] == t:
            p = top.xyz[top.edge_free[n, side]]
            return s * top.edge_len[n] / (2.0 * top.area[t]) * (r - p)
    return np.zeros_like(r)


def rwg_div(top: Topology, n: int, t: int) -> float:
    for side, s in ((0, 1.0), (1, -1.0)):
        if top.edge_tri[n, side] == t:
            return s * top.edge_len[n] / top.area[t]
    return 0.0


def local_coefficients(top: Topology, x):
    """Affine restriction of the expanded current to each triangle.

    For x = [x_J ; x_sigma] (mesh order), J|_t(r) = a_t (r - c_t) + beta_t with
    a_t = sum_n s l_n x_n / (2 A_t) and beta_t = J(c_t); sigma_t = x_sigma[t].
    Returns a [T], beta [T,3], sigma [T] (complex128).
    """
    E = top.E
    xJ = np.asarray(x[:E])
    xs = np.asarray(x[E:])
    T = top.T
    a = np.zeros(T, np.complex128)
    beta = np.zeros((T, 3), np.complex128)
    for t in range(T):
        for k in range(3):
            n = top.tri_edges[t, k]
            if n < 0:
                continue
            s = top.tri_sign[t, k]
            side = 0 if s > 0 else 1
            p = top.xyz[top.edge_free[n, side]]
            c = s * top.edge_len[n] / (2.0 * top.area[t])
            a[t] += c * xJ[n]
            beta[t] += c * xJ[n] * (top.centroid[t] - p)
    return a, beta, xs.astype(np.complex128)
