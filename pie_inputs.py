"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds geometry and random numbers only, none of the method's
arithmetic: triangulated PEC surfaces shaped like the paper's canonical
problems (the sphere of Section 4), complex excitation vectors drawn from a
seeded generator, and plane-wave directions.  Both the oracle and the product
path receive exactly these arrays.
"""
from __future__ import annotations

import itertools

import numpy as np


def icosahedron():
    """Regular icosahedron on the unit sphere.

    Vertices are the cyclic permutations of (0, +-1, +-phi), normalised.  Faces
    are the vertex triples whose three pairwise distances equal the edge
    length; each face is oriented so that its normal points away from the
    origin.
    """
    phi = (1.0 + np.sqrt(5.0)) / 2.0
    base = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            base.append((0.0, s1, s2 * phi))
            base.append((s1, s2 * phi, 0.0))
            base.append((s2 * phi, 0.0, s1))
    v = np.array(base, dtype=np.float64)
    edge2 = 4.0  # squared edge length of the unnormalised solid
    faces = []
    for i, j, k in itertools.combinations(range(12), 3):
        d = [np.sum((v[a] - v[b]) ** 2) for a, b in ((i, j), (j, k), (i, k))]
        if all(abs(x - edge2) < 1e-9 for x in d):
            n = np.cross(v[j] - v[i], v[k] - v[i])
            if np.dot(n, v[i] + v[j] + v[k]) < 0:
                faces.append((i, k, j))
            else:
                faces.append((i, j, k))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, np.array(faces, dtype=np.int32)


def icosphere(n: int, radius: float = 1.0):
    """Icosahedron subdivided n times (each triangle into 4 by edge midpoints),
    every new vertex projected onto the sphere of the given radius.

    Counts: T = 20*4**n, E = 30*4**n, V = 10*4**n + 2.  Returns
    (xyz float64 [V,3], tri int32 [T,3]) with outward (counter-clockwise)
    orientation.
    """
    v, f = icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(n):
        mid = {}
        newf = []

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                p = (np.array(verts[a]) + np.array(verts[b])) * 0.5
                p = p / np.linalg.norm(p)
                mid[key] = len(verts)
                verts.append(tuple(p))
            return mid[key]

        for a, b, c in f:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            newf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = np.array(newf, dtype=np.int32)
    xyz = np.array(verts, dtype=np.float64) * radius
    return xyz, np.ascontiguousarray(f, dtype=np.int32)


def flat_pair(shared: str = "edge"):
    """Two-triangle test meshes: coplanar pair sharing an edge, a folded pair
    sharing an edge (90 degrees), or two triangles sharing only a vertex."""
    if shared == "edge":
        xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], float) * 0.1
        tri = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    elif shared == "fold":
        xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.5, 0.2, 0.9]], float) * 0.1
        tri = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    elif shared == "vertex":
        xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0.2, 0.3], [-0.3, -1, 0.1]], float) * 0.1
        tri = np.array([[0, 1, 2], [0, 3, 4]], np.int32)
    else:
        raise ValueError(shared)
    return xyz, tri


def square_patch(n: int, side: float = 0.6):
    """Flat square plate of the given side in the x-y plane, centred at the
    origin: an n x n grid of squares, each split by its (+x,+y) diagonal into
    two triangles, normals along +z.  T = 2 n^2, interior edges 3 n^2 - 2 n.
    Returns (xyz [V,3], tri [T,3])."""
    g = np.linspace(-0.5 * side, 0.5 * side, n + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    tri = []
    for i in range(n):
        for j in range(n):
            a = i * (n + 1) + j
            b = (i + 1) * (n + 1) + j
            tri.append((a, b, b + 1))
            tri.append((a, b + 1, a + 1))
    return xyz, np.array(tri, dtype=np.int32)


class _VertexSet:
    """Vertices keyed by exact (integer or rational) labels, so that surfaces
    assembled face by face share their seam vertices."""

    def __init__(self):
        self.index = {}
        self.xyz = []

    def add(self, key, p):
        if key not in self.index:
            self.index[key] = len(self.xyz)
            self.xyz.append(p)
        return self.index[key]


def cube(n: int = 32, side: float = 1.0):
    """Closed cube centred at the origin: every face an n x n grid of squares,
    each square split by its two diagonals into 4 triangles around its centre
    (T = 24 n^2; n = 32 gives 24,576).  Outward orientation."""
    vs = _VertexSet()
    tri = []
    h = side / n
    for axis in range(3):
        for sgn in (-1, 1):
            u, v = [a for a in range(3) if a != axis]
            for i in range(n):
                for j in range(n):
                    def corner(ii, jj):
                        lab = [0, 0, 0]
                        lab[axis] = sgn * n
                        lab[u] = 2 * ii - n
                        lab[v] = 2 * jj - n
                        return vs.add(("g",) + tuple(lab), np.array(lab, float) * 0.5 * h)
                    a, b, c, d = corner(i, j), corner(i + 1, j), corner(i + 1, j + 1), corner(i, j + 1)
                    lab = [0, 0, 0]
                    lab[axis] = sgn * n
                    lab[u] = 2 * i + 1 - n
                    lab[v] = 2 * j + 1 - n
                    m = vs.add(("c",) + tuple(lab), np.array(lab, float) * 0.5 * h)
                    quad = [(a, b), (b, c), (c, d), (d, a)]
                    for p0, p1 in quad:
                        tri.append((p0, p1, m))
    xyz = np.array(vs.xyz)
    tri = np.array(tri, np.int64)
    # orient outward: normal . (centroid) > 0 (the cube is centred at the origin)
    v0, v1, v2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    flip = np.sum(np.cross(v1 - v0, v2 - v0) * (v0 + v1 + v2), axis=1) < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return xyz, tri.astype(np.int32)


def octasphere(n: int, axes=(1.0, 1.0, 1.0)):
    """Octahedron subdivided n times (midpoints projected to the unit sphere),
    then scaled to an ellipsoid with the given semi-axes: T = 8 * 4**n
    (n = 6: 32,768; axes (1, 0.5, 0.5) is the 2:1:1 prolate ellipsoid)."""
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    faces = []
    for sx in (0, 1):
        for sy in (2, 3):
            for sz in (4, 5):
                f = (sx, sy, sz)
                nrm = np.cross(v[f[1]] - v[f[0]], v[f[2]] - v[f[0]])
                faces.append(f if np.dot(nrm, v[sx] + v[sy] + v[sz]) > 0 else (sx, sz, sy))
    verts = [tuple(p) for p in v]
    f = np.array(faces)
    for _ in range(n):
        mid = {}
        newf = []

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                p = (np.array(verts[a]) + np.array(verts[b])) * 0.5
                mid[key] = len(verts)
                verts.append(tuple(p / np.linalg.norm(p)))
            return mid[key]

        for a, b, c in f:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            newf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = np.array(newf)
    xyz = np.array(verts) * np.asarray(axes, float)
    return xyz, f.astype(np.int32)


def cylinder(radius: float = 0.5, height: float = 2.0, nseg: int = 128, nrings: int = 20, nrows: int = 119):
    """Closed circular cylinder with flat caps, axis z, centred at the origin.
    Side: nrows rows of 2*nseg triangles; each cap: a fan of nseg triangles
    plus nrings annuli of 2*nseg triangles (defaults: 40,960 triangles).
    Outward orientation."""
    vs = _VertexSet()
    tri = []
    ang = 2 * np.pi * np.arange(nseg) / nseg

    def ring(z_label, r_label, z, r):
        return [vs.add(("r", z_label, r_label, k), np.array([r * np.cos(a), r * np.sin(a), z])) for k, a in enumerate(ang)]

    zs = np.linspace(-0.5 * height, 0.5 * height, nrows + 1)
    side = [ring(i, nrings + 1, zs[i], radius) for i in range(nrows + 1)]
    for i in range(nrows):
        lo, hi = side[i], side[i + 1]
        for k in range(nseg):
            k1 = (k + 1) % nseg
            tri.append((lo[k], lo[k1], hi[k1]))
            tri.append((lo[k], hi[k1], hi[k]))
    for cap, zi in ((0, 0), (1, nrows)):
        z = zs[zi]
        rings = [ring(zi, q, z, radius * q / (nrings + 1)) for q in range(1, nrings + 1)] + [side[zi]]
        centre = vs.add(("c", cap), np.array([0.0, 0.0, z]))
        first = rings[0]
        for k in range(nseg):
            tri.append((centre, first[k], first[(k + 1) % nseg]))
        for q in range(nrings):
            a, b = rings[q], rings[q + 1]
            for k in range(nseg):
                k1 = (k + 1) % nseg
                tri.append((a[k], b[k], b[k1]))
                tri.append((a[k], b[k1], a[k1]))
    xyz = np.array(vs.xyz)
    tri = np.array(tri, np.int64)
    v0, v1, v2 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    c = (v0 + v1 + v2) / 3.0
    out = np.where(np.abs(c[:, 2]) >= 0.5 * height - 1e-12, np.sign(c[:, 2]) * nrm[:, 2],
                   np.sum(nrm[:, :2] * c[:, :2], axis=1))
    flip = out < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return xyz, tri.astype(np.int32)


def complex_normal(shape, seed: int) -> np.ndarray:
    """Complex normal samples, real and imaginary parts each N(0,1), from
    numpy's PCG64 generator with the given seed (complex128)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im).astype(np.complex128)


def planewave_set():
    """The 64 plane waves of the batched and gradient workloads: propagation
    directions -r(theta, phi) on a uniform grid, theta at the midpoints of 4
    equal bands of [0, pi] and phi at 8 steps of pi/4, each with the theta
    and the phi polarisation.  Returns a list of (khat [3], pol [3])."""
    waves = []
    for t in (np.arange(4) + 0.5) * np.pi / 4:
        for p in np.arange(8) * 2 * np.pi / 8:
            kh = -np.array([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)])
            e_th = np.array([np.cos(t) * np.cos(p), np.cos(t) * np.sin(p), -np.sin(t)])
            e_ph = np.array([-np.sin(p), np.cos(p), 0.0])
            waves += [(kh, e_th), (kh, e_ph)]
    return waves


def bistatic_directions(n: int = 181, phi: float = 0.0) -> np.ndarray:
    """Unit directions in the x-z plane (azimuth phi) at polar angles
    theta = 0..180 degrees in n equal steps, [n,3] float64."""
    th = np.linspace(0.0, np.pi, n)
    return np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)], axis=1)
