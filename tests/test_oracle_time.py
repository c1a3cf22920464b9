"""Pins of the oracle's temporal part against what the paper fixes.

Sec. 3 (smooth step f, cutoffs f_i, bumps rho_i, partition of unity mu_i,
basis b_{i,m}, Eq. BasisFunctions), Eq. psis (psi, psi~), Sec. 3.1
(prototype shift invariance Eq. psiTildeRed, parity Eq. symmetryXi, swap
Eq. symmetryXip), Sec. 3.2 (support of psi).
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1503_07221_gb300 import inputs


def _tiny(t, p=0, **kw):
    V, F = inputs.tiny_meshes()["tetra"]
    return Oracle(V, F, t, p=p, equidistant=False, psi_mode="direct", **kw)


@pytest.fixture(scope="module")
def eq9():
    return _tiny(inputs.equidistant_grid(9, 2.0))


def test_step_function_values(eq9):
    # b_1 = 8 mu_1 (t/dt)^2 P_0 with mu_1 = 1 - f_0 and f_0(dt/2) = f(0) = 1/2
    dt = 0.25
    v = eq9.basis(0, 0, np.array([dt / 2]))[0, 0]
    assert abs(v - 1.0) < 1e-15
    # inner bump at its centre equals 1, at the ends 0 (Sec. 3: rho_i)
    mu = eq9.mu(3, np.array([3 * dt, 2 * dt, 4 * dt, 2.5 * dt, 3.5 * dt]))[:, 0]
    assert abs(mu[0] - 1.0) < 1e-15 and mu[1] == 0.0 and mu[2] == 0.0
    # symmetry f(-x) = 1 - f(x): the rising and falling halves mirror
    assert abs(mu[3] - mu[4]) < 1e-15 and abs(mu[3] - 0.5) < 1e-15
    # f(x) = erf(2 artanh x)/2 + 1/2 at x = 1/2 on the rising flank of mu_4
    x = 0.5
    s = 2 * dt + (x + 1) / 2 * dt
    want = 0.5 * math.erf(2 * math.atanh(x)) + 0.5
    assert abs(eq9.mu(3, np.array([s]))[0, 0] - want) < 1e-15


@pytest.mark.parametrize("grid", ["eq", "graded"])
def test_partition_of_unity(grid):
    t = inputs.equidistant_grid(9, 2.0) if grid == "eq" else inputs.graded_grid(12, 1.1, 3.0)
    o = _tiny(t)
    o.set_first_kind(1)  # mu_1 instead of b_1 = 8 mu_1 (t/dt)^2
    s = np.linspace(0.0, t[-1], 4001)
    tot = sum(o.mu(i, s)[:, 0] for i in range(t.size))
    assert np.abs(tot - 1.0).max() < 1e-15
    b = sum(o.basis(i, 0, s)[:, 0] for i in range(t.size))
    assert np.abs(b - 1.0).max() < 1e-15
    # derivatives of the sum vanish away from t = 0
    d1 = sum(o.basis(i, 0, s[1:])[:, 1] for i in range(t.size))
    d2 = sum(o.basis(i, 0, s[1:])[:, 2] for i in range(t.size))
    assert np.abs(d1).max() < 1e-9 and np.abs(d2).max() < 1e-6 * np.abs(o.basis(2, 0, s)[:, 2]).max()


@pytest.mark.parametrize("grid", ["eq", "graded"])
def test_supports(grid):
    t = inputs.equidistant_grid(9, 2.0) if grid == "eq" else inputs.graded_grid(12, 1.1, 3.0)
    o = _tiny(t)
    N = t.size
    s = np.linspace(-0.5, t[-1], 6001)
    for i in range(N):
        v = o.mu(i, s)[:, 0]
        lo = 0.0 if i == 0 else t[i - 1]
        hi = t[-1] + 1 if i == N - 1 else t[i + 1]
        inside = (s > lo) & (s < hi) if i > 0 else (s >= 0) & (s < hi)
        assert np.all(v[~inside] == 0.0)
        strict = inside & (s > lo + 1e-9) & (s < hi - 1e-9)
        assert np.all(v[strict] > 0.0)


@pytest.mark.parametrize("ib,m", [(0, 0), (0, 1), (3, 0), (3, 2), (8, 1)])
def test_basis_derivatives_fd(eq9, ib, m):
    o = _tiny(inputs.equidistant_grid(9, 2.0), p=2)
    lo = 0.0 if ib == 0 else (ib - 1) * 0.25
    hi = min(2.0, (ib + 1) * 0.25)
    s = np.linspace(lo + 0.01, hi - 0.01, 37)
    s = s[np.abs(s - ib * 0.25) > 0.01]
    h = 1e-5
    v = o.basis(ib, m, s)
    vp = o.basis(ib, m, s + h)
    vm = o.basis(ib, m, s - h)
    fd1 = (vp[:, 0] - vm[:, 0]) / (2 * h)
    fd2 = (vp[:, 1] - vm[:, 1]) / (2 * h)
    sc1 = np.abs(v[:, 1]).max() + 1
    sc2 = np.abs(v[:, 2]).max() + 1
    assert np.abs(fd1 - v[:, 1]).max() < 1e-6 * sc1
    assert np.abs(fd2 - v[:, 2]).max() < 1e-6 * sc2


def test_legendre_factor(eq9):
    # b_{i,m} = mu_i P_m((t - t_{i-2})/dt - 1): at the bump centre P_m(0)
    o = _tiny(inputs.equidistant_grid(9, 2.0), p=2)
    c = 4 * 0.25
    assert abs(o.basis(4, 1, np.array([c]))[0, 0]) < 1e-15           # P_1(0) = 0
    assert abs(o.basis(4, 2, np.array([c]))[0, 0] + 0.5) < 1e-15     # P_2(0) = -1/2
    x = 0.3
    s = c + x * 0.25
    mu = o.mu(4, np.array([s]))[0, 0]
    assert abs(o.basis(4, 2, np.array([s]))[0, 0] - mu * 0.5 * (3 * x * x - 1)) < 1e-15


def _support(t, kb, ib):
    N = t.size
    tl = lambda q: 0.0 if q == 0 else t[q - 1]
    tr = lambda q: t[-1] if q == N - 1 else t[q + 1]
    return max(0.0, tl(kb) - tr(ib)), tr(kb) - tl(ib)


def test_psi_support(eq9):
    t = inputs.equidistant_grid(9, 2.0)
    for kb, ib in [(0, 0), (1, 0), (4, 2), (4, 5), (8, 3), (8, 8), (7, 8), (8, 0)]:
        a, b = _support(t, kb, ib)
        r = np.linspace(0.0, 2.5, 501)
        v = eq9.psi(kb, ib, r)
        out = ((r <= a) & (a > 0)) | (r >= b)
        assert np.all(v[out] == 0.0), (kb, ib)
        inn = (r > a + 1e-2) & (r < b - 1e-2)
        assert np.any(np.abs(v[inn, 1]) > 1e-8), (kb, ib)
    # block Hessenberg: psi vanishes identically when t_k <= t_{i-2} (Sec. 3.2)
    r = np.linspace(0.0, 2.0, 101)
    assert np.all(eq9.psi(2, 4, r) == 0.0)


@pytest.mark.parametrize("kb,ib", [(4, 2), (5, 0), (8, 3), (3, 4), (1, 1)])
def test_psi_is_second_derivative_of_psi_tilde(eq9, kb, ib):
    # b''_i(t-r) = d^2/dr^2 b_i(t-r), so psi = d^2 psi~/dr^2 (Eq. psis)
    t = inputs.equidistant_grid(9, 2.0)
    a, b = _support(t, kb, ib)
    r = np.linspace(a + 0.013, b - 0.013, 23)
    h = 2e-4
    v = eq9.psi(kb, ib, r)
    fd = (eq9.psi(kb, ib, r + h)[:, 1] - 2 * v[:, 1] + eq9.psi(kb, ib, r - h)[:, 1]) / h ** 2
    assert np.abs(fd - v[:, 0]).max() < 1e-4 * np.abs(v[:, 0]).max()


@pytest.mark.parametrize("grid", ["eq", "graded"])
def test_psi_partition_identity(grid):
    # Sum_i b_i(s) = 1 on [0,T] and 0 for s < 0, hence for an inner test
    # function: Sum_i psi~_{k,i}(r) = int_r^T b'_k = -b_k(r) and
    # Sum_i psi_{k,i}(r) = 0 for r > 0 (classical part).
    t = inputs.equidistant_grid(9, 2.0) if grid == "eq" else inputs.graded_grid(10, 1.15, 2.0)
    o = _tiny(t)
    o.set_first_kind(1)
    N = t.size
    r = np.linspace(0.003, t[-1] - 0.003, 97)
    for kb in [1, 3, N - 2]:
        s = sum(o.psi(kb, ib, r) for ib in range(N))
        bk = o.basis(kb, 0, r)[:, 0]
        assert np.abs(s[:, 1] + bk).max() < 1e-13
        scale = max(np.abs(o.psi(kb, ib, r)[:, 0]).max() for ib in range(N))
        assert np.abs(s[:, 0]).max() < 1e-12 * scale
    # last test function: b_N(T) = 1
    s = sum(o.psi(N - 1, ib, r) for ib in range(N))
    assert np.abs(s[:, 1] - (1.0 - o.basis(N - 1, 0, r)[:, 0])).max() < 1e-13


def test_prototype_shift_and_parity():
    # inner blocks depend on r + t_{i-2} - t_{k-2} only (Eq. psiTildeRed), and
    # the prototype has parity (-1)^{m1+m2+1} (Eq. symmetryXi)
    t = inputs.equidistant_grid(11, 2.5)
    dt = 0.25
    o = _tiny(t, p=1)
    al = np.linspace(0.01, 2 * dt - 0.01, 17)
    for m2 in range(2):
        for m1 in range(2):
            base = None
            for kb, ib in [(5, 3), (6, 4), (8, 6)]:
                d = (kb - ib) * dt
                v = o.psi(kb, ib, d + al, m2=m2, m1=m1)
                w = o.psi(kb, ib, d - al, m2=m2, m1=m1)
                sgn = (-1) ** (m1 + m2 + 1)
                sc = np.abs(v).max(axis=0)
                assert np.all(np.abs(v - sgn * w).max(axis=0) < 1e-13 * sc)
                if base is None:
                    base = v
                else:
                    assert np.all(np.abs(v - base).max(axis=0) < 1e-13 * sc)
    # swap symmetry: xi~_{m1,m2}(-a) = -xi~_{m2,m1}(a) (Eq. symmetryXip)
    kb, ib = 6, 4
    d = 2 * dt
    for m1, m2 in [(0, 1), (1, 0), (1, 1), (0, 0)]:
        v = o.psi(kb, ib, d - al, m2=m2, m1=m1)
        w = o.psi(kb, ib, d + al, m2=m1, m1=m2)
        sc = np.abs(v).max(axis=0)
        assert np.all(np.abs(v + w).max(axis=0) < 1e-13 * sc)


def test_graded_grid_breaks_shift_invariance():
    t = inputs.graded_grid(12, 1.1, 3.0)
    o = _tiny(t)
    al = np.linspace(0.01, 0.1, 9)
    v = o.psi(6, 4, t[5] - t[3] + al)
    w = o.psi(7, 5, t[6] - t[4] + al)
    assert np.abs(v - w).max() > 1e-3 * np.abs(v).max()


def test_quadrature_refinement_converged():
    t = inputs.equidistant_grid(9, 2.0)
    o1 = _tiny(t, gl_n=32, gl_sub=4)
    o2 = _tiny(t, gl_n=48, gl_sub=8)
    r = np.linspace(0.001, 1.9, 101)
    for kb, ib in [(0, 0), (3, 1), (5, 0), (8, 2), (8, 8), (7, 8)]:
        a = o1.psi(kb, ib, r)
        b = o2.psi(kb, ib, r)
        assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300), (kb, ib)


@pytest.mark.parametrize("t", [inputs.equidistant_grid(9, 2.0), inputs.graded_grid(8, 1.3, 2.0)],
                         ids=["eq", "graded"])
def test_interpolant_matches_direct(t):
    # on the graded grid the panel breakpoints t_{k-a} - t_{i-b} are all distinct
    V, F = inputs.tiny_meshes()["octa"]
    od = Oracle(V, F, t, equidistant=False, psi_mode="direct")
    oi = Oracle(V, F, t, equidistant=False, psi_mode="interp")
    r = np.random.default_rng(0).uniform(0.0, 2.0, 400)
    for blk in range(od.num_blocks()):
        a = od.psi_block(blk, r)
        b = oi.psi_block(blk, r)
        sc = np.abs(a).max(axis=0) + 1e-300
        assert np.all(np.abs(a - b).max(axis=0) <= 1e-11 * sc), blk
