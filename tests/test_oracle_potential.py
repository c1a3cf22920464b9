"""Pins of the oracle's retarded double layer potential u = D phi (Eq.
RetardedPotential), the evaluation of the solution off the surface.

* Gauss's law: for a density equal to 1 at every point and every time s >= 0
  (the partition of unity with mu_1 as the first time function, Sec. 3),
  d_t phi = 0 and, once every retarded time t - |x - y| is >= 0, u(x) =
  -1/(4 pi) int n_y.(x - y)/|x - y|^3 = 0 outside the closed surface and 1
  inside it (the solid angle). Before the first retarded time reaches
  the surface, u = 0 (causality).
* Unit sphere, density U(t) constant in space: with chord r from a point at
  distance R > 1 from the centre, dGamma_y = 2 pi r dr / R and
  n_y.(x - y) = (R^2 - 1 - r^2) / 2, so
      u(R, t) = -1/(4R) int_{R-1}^{R+1} (R^2 - 1 - r^2) [U(t - r)/r^2 + U'(t - r)/r] dr,
  a 1-D integral; the flat-triangle mesh approaches it at O(h^2).
"""
import numpy as np

from oracle.oracle import Oracle, gauss_legendre
from paper_1503_07221_gb300 import inputs

T9 = inputs.equidistant_grid(9, 2.0)


def test_gauss_law_and_causality():
    V, F = inputs.icosphere(2)
    o = Oracle(V, F, T9, psi_mode="direct")
    o.set_first_kind(1)  # time functions mu_1..mu_N: sum 1 for every s >= 0
    alpha = np.ones((o.L, o.M))
    X = np.array([[0, 0, 1.5], [0.3, -1.2, 0.9], [0, 0, 0.2], [0.1, 0.3, -0.4]])
    inside = np.array([0, 0, 1, 1])
    u = o.double_layer(alpha, X, [3.0], n=8)[:, 0]  # 3.0 > every |x - y| here
    assert np.abs(u - inside).max() < 1e-10
    # exterior points at distance >= 0.5 from the unit sphere (the mesh lies inside it)
    u0 = o.double_layer(alpha, X[:2], [0.45], n=8)
    assert np.array_equal(u0, np.zeros_like(u0))


def _reduced(U, R, t, grid):
    g, w = gauss_legendre(40)
    cuts = sorted({R - 1.0, R + 1.0} | {t - x for x in grid if R - 1.0 < t - x < R + 1.0})
    tot = 0.0
    for a, b in zip(cuts[:-1], cuts[1:]):
        r = a + (b - a) * g
        v = U(t - r)
        tot += np.sum((b - a) * w * (R * R - 1.0 - r * r) * (v[:, 0] / r ** 2 + v[:, 1] / r))
    return -tot / (4.0 * R)


def test_sphere_constant_density_reduction():
    a = np.random.default_rng(4).standard_normal(T9.size)
    X = np.array([[0, 0, 1.5], [1.2, 0.9, 1.0]])
    times = [1.0, 2.2, 3.1]
    err = []
    for level in (2, 3):
        V, F = inputs.icosphere(level)
        o = Oracle(V, F, T9, psi_mode="direct")
        U = lambda s: sum(a[k] * o.basis(k, 0, np.atleast_1d(s))[:, :2] for k in range(T9.size))
        ex = np.array([[_reduced(U, np.linalg.norm(x), t, T9) for t in times] for x in X])
        u = o.double_layer(np.repeat(a[:, None], o.M, axis=1), X, times, n=8)
        err.append(np.abs(u - ex).max() / np.abs(ex).max())
    # measured 0.058, 0.016 (and 0.0037 on 5120 triangles)
    assert err[1] <= 0.03 and err[1] * 3.0 <= err[0], err
