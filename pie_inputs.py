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


def complex_normal(shape, seed: int) -> np.ndarray:
    """Complex normal samples, real and imaginary parts each N(0,1), from
    numpy's PCG64 generator with the given seed (complex128)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im).astype(np.complex128)


def balanced_vector(n_rwg: int, n_tri: int, seed: int, sigma_scale: float) -> np.ndarray:
    """Complex normal excitation vector in mesh order [RWG ; pulse], with the
    pulse part multiplied by sigma_scale so that both blocks of the operator
    contribute at comparable magnitude."""
    x = complex_normal(n_rwg + n_tri, seed)
    x[n_rwg:] *= sigma_scale
    return x


def bistatic_directions(n: int = 181, phi: float = 0.0) -> np.ndarray:
    """Unit directions in the x-z plane (azimuth phi) at polar angles
    theta = 0..180 degrees in n equal steps, [n,3] float64."""
    th = np.linspace(0.0, np.pi, n)
    return np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)], axis=1)
