"""Pins of the oracle's right-hand side g_k(l) = int int g phi_l bdot_k
(Sec. 3, the vector of the linear system) and of its dense solve.

* Space-independent and linear-in-space data (the sphere tests of Sec. 6.1):
  the spatial integrals of the hat functions are closed forms
  (int_T lambda_a = |T|/3, int_T lambda_a lambda_b = |T| (1 + delta_ab)/12),
  and the time integral is recomputed with scipy's adaptive quadrature.
* Plane-wave data: brute force on one small triangle with a collapsed
  tensor Gauss rule (not the 7-point rule) and a fine time rule.
* Dense solve: the oracle's LU solution satisfies the reduced block system
  through hessenberg_apply (itself pinned against the full block list).
"""
import numpy as np
import pytest
from scipy.integrate import quad

from oracle.oracle import Oracle, Y00, Y10, g_data, g_time
from paper_1503_07221_gb300 import inputs


def _time_integral(o, k, f):
    t = o.t
    a = 0.0 if k == 0 else t[k - 1]
    b = t[-1] if k == o.N - 1 else t[k + 1]
    pts = [x for x in t if a < x < b]
    bd = lambda s: float(o.basis(k, 0, np.array([s]))[0, 1])
    return quad(lambda s: f(s) * bd(s), a, b, points=pts or None, limit=200, epsabs=1e-13, epsrel=1e-12)[0]


def _areas(V, F):
    P = V[F]
    return 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)


def test_rhs_sphere_n0_closed_form():
    V, F = inputs.icosphere(1)
    o = Oracle(V, F, inputs.equidistant_grid(9, 2.0))
    g = o.rhs(1)
    A = _areas(V, F)
    w = np.zeros(o.M)
    np.add.at(w, F.ravel(), np.repeat(A / 3.0, 3))
    for k in range(o.N):
        tk = Y00 * _time_integral(o, k, lambda s: float(g_time(1, s)))
        ref = w * tk
        assert np.abs(g[k] - ref).max() <= 1e-10 * max(np.abs(ref).max(), 1e-300), k


def test_rhs_sphere_n1_closed_form():
    V, F = inputs.icosphere(1)
    o = Oracle(V, F, inputs.equidistant_grid(9, 2.0))
    g = o.rhs(2)
    A = _areas(V, F)
    z = V[:, 2]
    w = np.zeros(o.M)
    for e in range(F.shape[0]):
        zs = z[F[e]]
        for a in range(3):
            w[F[e, a]] += A[e] / 12.0 * (zs.sum() + zs[a])
    for k in range(o.N):
        tk = Y10 * _time_integral(o, k, lambda s: float(g_time(2, s)))
        ref = w * tk
        assert np.abs(g[k] - ref).max() <= 1e-10 * np.abs(ref).max() + 1e-16, k


def test_rhs_plane_wave_brute_force():
    # one triangle of diameter ~0.05 near (0, 0, 1); pulse c0 = 0.5, w = 0.2
    V = np.array([[0.0, 0.0, 1.0], [0.04, 0.0, 0.99], [0.0, 0.05, 0.995]])
    F = np.array([[0, 1, 2]], dtype=np.int32)
    t = inputs.equidistant_grid(6, 2.0)
    prm = (0.3, -0.2, 0.9, 0.5, 0.2)
    d = np.array(prm[:3]) / np.linalg.norm(prm[:3])
    prm_n = tuple(d) + prm[3:]
    o = Oracle(V, F, t)
    g = o.rhs(0, prm_n)
    n = np.cross(V[1] - V[0], V[2] - V[0])
    area = 0.5 * np.linalg.norm(n)
    n = n / np.linalg.norm(n)
    # collapsed Gauss on the unit triangle: (u, v) = (x, y (1 - x))
    xg, wg = np.polynomial.legendre.leggauss(24)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    U, W = [], []
    for i in range(24):
        for j in range(24):
            U.append((xg[i], xg[j] * (1 - xg[i])))
            W.append(wg[i] * wg[j] * (1 - xg[i]))
    U, W = np.array(U), np.array(W) * 2.0  # reference area 1/2 -> weights sum to 1
    lam = np.stack([1 - U[:, 0] - U[:, 1], U[:, 0], U[:, 1]], axis=1)
    X = lam @ V
    ts = np.concatenate([a + (b - a) * (np.polynomial.legendre.leggauss(40)[0] + 1) / 2
                         for a, b in zip(t[:-1], t[1:])])
    wt = np.concatenate([(b - a) / 2 * np.polynomial.legendre.leggauss(40)[1] for a, b in zip(t[:-1], t[1:])])
    G = g_data(0, prm_n, X, np.repeat(n[None], len(X), axis=0), ts)  # (P, T)
    for k in range(o.N):
        bd = o.basis(k, 0, ts)[:, 1]
        Ht = G @ (wt * bd)
        for a in range(3):
            ref = area * np.sum(W * lam[:, a] * Ht)
            assert abs(g[k, F[0, a]] - ref) <= 1e-9 * np.abs(g).max(), (k, a, g[k, F[0, a]], ref)


def test_dense_solve_satisfies_reduced_system():
    V, F = inputs.icosphere(1)
    o = Oracle(V, F, inputs.equidistant_grid(9, 2.0))
    g = o.rhs(0, (0.0, 0.0, 1.0, 2.0, 0.2))
    alpha = o.solve_dense(g)
    r = o.hessenberg_apply(alpha) - g
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(g)
