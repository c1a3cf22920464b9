"""Seeded synthetic inputs: surface meshes and time grids.

This module holds no arithmetic of the space-time Galerkin method itself. It
only builds the geometry and the time grid that both the CUDA path and the CPU
oracle consume as input data:

* icosphere(level)           -- flat-triangle unit sphere, 20*4**level triangles,
                                outward (counter-clockwise) orientation
* torus(R, r, n_major, n_minor) -- quad grid split into triangles, outward
* jitter(verts, tris, frac, seed) -- per-vertex uniform displacement in
                                [-frac*h, frac*h]^3, h = mean edge length,
                                drawn from a splitmix64 stream
* equidistant_grid(N, T)     -- t_i = i*T/(N-1), i = 0..N-1 (Sec. 3: N points)
* graded_grid(steps, q, T)   -- dt_n = dt_0*q**n, n = 0..steps-1, summing to T

The named workloads (sphere 320 / 5120 jittered / 20480, torus 8192 graded)
are assembled by `workload(name)`, the potential evaluations (points on a
plane, grid times) by `potential_workload(name)`.
"""
from __future__ import annotations

import dataclasses
import numpy as np

_MASK64 = (1 << 64) - 1


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the splitmix64 sequence started at `seed`.

    splitmix64 (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15, then
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) *
    0x94D049BB133111EB; z ^= z >> 31. The top 53 bits give the double.
    """
    out = np.empty(n, dtype=np.float64)
    state = seed & _MASK64
    for k in range(n):
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        z = z ^ (z >> 31)
        out[k] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out


def icosphere(level: int):
    """Unit icosphere with 20*4**level flat triangles and 10*4**level+2 vertices.

    Each refinement splits a triangle into four through its edge midpoints;
    new vertices are projected onto the unit sphere. Triangles are listed
    counter-clockwise seen from outside (outward normal)."""
    p = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
         (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    verts = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.ascontiguousarray(np.array(verts, dtype=np.float64))
    F = np.ascontiguousarray(np.array(faces, dtype=np.int32))
    _orient_outward(V, F)
    return V, F


def torus(R: float = 1.0, r: float = 0.4, n_major: int = 128, n_minor: int = 32):
    """Torus (R, r) from an n_major x n_minor quad grid, two triangles per quad,
    outward orientation: 2*n_major*n_minor triangles, n_major*n_minor vertices."""
    u = 2.0 * np.pi * np.arange(n_major) / n_major
    w = 2.0 * np.pi * np.arange(n_minor) / n_minor
    U, W = np.meshgrid(u, w, indexing="ij")
    X = (R + r * np.cos(W)) * np.cos(U)
    Y = (R + r * np.cos(W)) * np.sin(U)
    Z = r * np.sin(W)
    V = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    idx = lambda i, j: (i % n_major) * n_minor + (j % n_minor)
    F = []
    for i in range(n_major):
        for j in range(n_minor):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            F.append((a, b, c))
            F.append((a, c, d))
    V = np.ascontiguousarray(V)
    F = np.ascontiguousarray(np.array(F, dtype=np.int32))
    _orient_outward_torus(V, F, R)
    return V, F


def _orient_outward(V, F):
    """Flip triangles whose normal points towards the origin (star-shaped)."""
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, a + b + c) < 0
    F[flip] = F[flip][:, [0, 2, 1]]


def _orient_outward_torus(V, F, R):
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    ring = cen.copy()
    ring[:, 2] = 0.0
    ring *= (R / np.linalg.norm(ring, axis=1))[:, None]
    flip = np.einsum("ij,ij->i", n, cen - ring) < 0
    F[flip] = F[flip][:, [0, 2, 1]]


def mean_edge_length(V, F) -> float:
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return float(np.linalg.norm(V[e[:, 0]] - V[e[:, 1]], axis=1).mean())


def jitter(V, F, frac: float = 0.01, seed: int = 0):
    """Displace every vertex by a uniform vector in [-frac*h, frac*h]^3."""
    h = mean_edge_length(V, F)
    u = splitmix64_uniform(seed, V.shape[0] * 3).reshape(V.shape)
    return np.ascontiguousarray(V + (2.0 * u - 1.0) * frac * h)


def equidistant_grid(N: int, T: float) -> np.ndarray:
    """N grid points t_i = i*T/(N-1) (the paper's N counts points, Sec. 3)."""
    return np.ascontiguousarray(np.arange(N, dtype=np.float64) * (T / (N - 1)))


def graded_grid(steps: int, q: float, T: float) -> np.ndarray:
    """steps+1 points with geometric step widths dt_n = dt_0 q**n summing to T."""
    dt0 = T * (q - 1.0) / (q ** steps - 1.0)
    t = np.concatenate([[0.0], np.cumsum(dt0 * q ** np.arange(steps))])
    t[-1] = T
    return np.ascontiguousarray(t)


@dataclasses.dataclass
class Workload:
    name: str
    verts: np.ndarray
    tris: np.ndarray
    t: np.ndarray
    equidistant: bool
    p: int = 0
    c: float = 1.0
    note: str = ""

    @property
    def M(self):
        return self.verts.shape[0]

    @property
    def E(self):
        return self.tris.shape[0]

    @property
    def N(self):
        return self.t.shape[0]


def workload(name: str) -> Workload:
    """Named synthetic workloads.

    sphere320   : icosphere level 2 (320 / 162), N=17 points, dt=0.25, T=4
    sphere5120j : icosphere level 4 (5120 / 2562) jittered +-1% h (seed 0),
                  N=65, dt=0.0625, T=4
    torus8192g  : torus R=1 r=0.4 (128x32 quads, 8192 / 4096), graded grid of
                  96 steps, ratio 1.02, on [0, 6]
    torus2048g  : the same torus and grid on 64x16 quads (2048 / 1024), a
                  small case of the same kernels (profiling, parity)
    sphere20480 : icosphere level 5 (20480 / 10242), N=129, dt=0.05, T=6.4
    sphere5120p : icosphere level 4 (5120 / 2562), N=65, dt=0.07, T=4.48: a
                  small case of the 20480 sphere's far-kernel shape (the 7
                  points of a triangle span less than one time step, as
                  there), for profiling
    """
    if name == "sphere320":
        V, F = icosphere(2)
        return Workload(name, V, F, equidistant_grid(17, 4.0), True)
    if name == "sphere5120j":
        V, F = icosphere(4)
        return Workload(name, jitter(V, F, 0.01, 0), F, equidistant_grid(65, 4.0), True)
    if name == "torus8192g":
        V, F = torus(1.0, 0.4, 128, 32)
        return Workload(name, V, F, graded_grid(96, 1.02, 6.0), False)
    if name == "torus2048g":
        V, F = torus(1.0, 0.4, 64, 16)
        return Workload(name, V, F, graded_grid(96, 1.02, 6.0), False)
    if name == "sphere20480":
        V, F = icosphere(5)
        return Workload(name, V, F, equidistant_grid(129, 6.4), True)
    if name == "sphere5120p":
        V, F = icosphere(4)
        return Workload(name, V, F, equidistant_grid(65, 4.48), True)
    raise KeyError(name)


@dataclasses.dataclass
class PotentialWorkload:
    """Evaluation of the retarded double layer potential off the surface: a
    mesh and time grid (the density lives on them), points X (P, 3), times
    (nt,) and the Gauss points per direction n of the collapsed rule."""
    name: str
    verts: np.ndarray
    tris: np.ndarray
    t: np.ndarray
    X: np.ndarray
    times: np.ndarray
    n: int


def plane_points(side: int, half: float, z: float) -> np.ndarray:
    """side x side grid of points on [-half, half]^2 at height z, x fastest."""
    g = np.linspace(-half, half, side)
    yy, xx = np.meshgrid(g, g, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), np.full(side * side, z)], axis=1)


def potential_workload(name: str) -> PotentialWorkload:
    """Named potential evaluations.

    plane66049_sphere320 : 257 x 257 = 66049 points on the plane z = 0.05
                           over [-3, 3]^2 (it cuts the sphere), the 40 grid
                           times t_1..t_40 of N = 41 points on [0, 6], the
                           320-triangle icosphere, 4 x 4 Gauss points per
                           triangle
    plane4096_sphere5120 : 64 x 64 points on the same plane, the same times,
                           the 5120-triangle icosphere, 4 x 4 points
    """
    t = equidistant_grid(41, 6.0)
    if name == "plane66049_sphere320":
        V, F = icosphere(2)
        return PotentialWorkload(name, V, F, t, plane_points(257, 3.0, 0.05), t[1:].copy(), 4)
    if name == "plane4096_sphere5120":
        V, F = icosphere(4)
        return PotentialWorkload(name, V, F, t, plane_points(64, 3.0, 0.05), t[1:].copy(), 4)
    raise KeyError(name)


def tiny_meshes():
    """Hand-built meshes of 2-20 triangles for brute-force checks."""
    out = {}
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], dtype=np.float64) * 0.5
    out["coplanar2"] = (V, np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32))
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0.6]], dtype=np.float64) * 0.5
    out["bent2"] = (V, np.array([[0, 1, 2], [1, 3, 2]], dtype=np.int32))
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) * 0.4
    F = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], dtype=np.int32)
    _orient_outward(V, F)
    out["tetra"] = (V, F)
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                 dtype=np.float64) * 0.5
    F = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                  [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], dtype=np.int32)
    _orient_outward(V, F)
    out["octa"] = (V, F)
    V, F = icosphere(0)
    out["icosa"] = (V * 0.5, F)
    return out
