"""Pins of the oracle's spatial quadrature, geometry, culling and assembled
blocks against closed forms and properties the paper fixes.

Eq. MatrixEntries (the element-pair integrand), Eq. SparsitySmallBlock
(mindist / maxdist culling), Sec. 3.2 (block Hessenberg form, Eq.
relationAtildeBlock block-Toeplitz reuse, the lag cutoff by diam), Sec. 5.1
(unique-block list and the count n_z of inner nonzero blocks), Sec. 2
(surface curl), Sec. 6.1 (unit sphere).
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, gauss_legendre, rule7, ss_rule
from paper_1503_07221_gb300 import inputs


# ----------------------------------------------------------------- rules --
def _tri_monomial(a, b):
    # int over {0 <= x2 <= x1 <= 1} of x1^a x2^b
    return 1.0 / ((b + 1) * (a + b + 2))


def test_gauss_legendre_exact():
    for n in (1, 2, 4, 7, 16):
        x, w = gauss_legendre(n)
        for k in range(2 * n):
            assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14


def test_rule7_degree5():
    bary, w = rule7()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(bary.sum(axis=1), 1.0, atol=1e-15)
    # on the unit right triangle (0,0),(1,0),(0,1): int x^a y^b = a! b! / (a+b+2)!
    x, y = bary[:, 1], bary[:, 2]
    for a in range(6):
        for b in range(6 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs(0.5 * np.sum(w * x ** a * y ** b) - exact) < 1e-15
    # degree 6 is not integrated exactly
    assert abs(0.5 * np.sum(w * x ** 6) - math.factorial(6) / math.factorial(8)) > 1e-6


@pytest.mark.parametrize("kase,count", [(3, 6), (2, 5), (1, 2)])
def test_sauter_schwab_polynomials(kase, count):
    n = 6
    xh, yh, w = ss_rule(kase, n)
    assert xh.shape[0] == count * n ** 4
    for a, b, c, d in [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 1, 0), (2, 1, 0, 2), (1, 1, 1, 1), (3, 0, 0, 2)]:
        s = np.sum(w * xh[:, 0] ** a * xh[:, 1] ** b * yh[:, 0] ** c * yh[:, 1] ** d)
        assert abs(s - _tri_monomial(a, b) * _tri_monomial(c, d)) < 1e-13
    # points lie in the reference triangle
    for P in (xh, yh):
        assert np.all(P[:, 1] >= -1e-15) and np.all(P[:, 1] <= P[:, 0] + 1e-15) and np.all(P[:, 0] <= 1 + 1e-15)


def _potential_in_plane(P, A, B, C):
    """int over triangle ABC of 1/|x-P| for P in its plane (polar integration
    around P: sum over edges of d_e [asinh(s+/d_e) - asinh(s-/d_e)])."""
    n = np.cross(B - A, C - A)
    n = n / np.linalg.norm(n)
    tot = 0.0
    for U, W in ((A, B), (B, C), (C, A)):
        e = W - U
        L = np.linalg.norm(e)
        e = e / L
        m = np.cross(e, n)  # outward in-plane normal of a CCW edge
        d = np.dot(U - P, m)
        if abs(d) < 1e-14:
            continue
        s0 = np.dot(U - P, e)
        s1 = s0 + L
        tot += d * (math.asinh(s1 / abs(d)) - math.asinh(s0 / abs(d)))
    return tot


def _outer(P3, fun, n):
    # collapsed Gauss product rule on triangle P3 (integrates fun over it)
    x, w = np.polynomial.legendre.leggauss(n)
    x = 0.5 * (x + 1)
    w = 0.5 * w
    A, B, C = P3
    area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
    s = 0.0
    for i in range(n):
        for j in range(n):
            u, v = x[i], x[j]
            b = np.array([1 - u, u * (1 - v), u * v])
            s += 2 * u * w[i] * w[j] * fun(b[0] * A + b[1] * B + b[2] * C)
    return s * area


def _ss_laplace(X, Y, kase, n):
    """int_X int_Y 1/|x-y| with the oracle's Sauter-Schwab rule; X, Y ordered so
    the shared vertices come first in the same order."""
    xh, yh, w = ss_rule(kase, n)
    def to3(P, h):
        return P[0][None] + h[:, :1] * (P[1] - P[0])[None] + h[:, 1:] * (P[2] - P[1])[None]
    x = to3(X, xh)
    y = to3(Y, yh)
    jx = np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))
    jy = np.linalg.norm(np.cross(Y[1] - Y[0], Y[2] - Y[0]))
    return jx * jy * np.sum(w / np.linalg.norm(x - y, axis=1))


@pytest.mark.parametrize("kase", [3, 2, 1])
def test_sauter_schwab_singular_laplace(kase):
    # coplanar configurations: identical / common edge / common vertex
    A = np.array([0.0, 0.0, 0.0]); B = np.array([1.0, 0.1, 0.0]); C = np.array([0.3, 0.9, 0.0])
    if kase == 3:
        X = Y = (A, B, C)
    elif kase == 2:
        D = np.array([1.2, -0.8, 0.0])
        X, Y = (A, B, C), (A, B, D)
    else:
        D = np.array([-0.9, -0.3, 0.0]); E = np.array([-0.2, -1.0, 0.0])
        X, Y = (A, B, C), (A, D, E)
    ref = _outer(X, lambda p: _potential_in_plane(p, *Y), 48)
    e4 = abs(_ss_laplace(X, Y, kase, 4) - ref) / ref
    e8 = abs(_ss_laplace(X, Y, kase, 8) - ref) / ref
    assert e8 < 1e-6 and e4 < 2e-3 and e8 < e4


def test_potential_formula_sanity():
    # far from the triangle the potential tends to area / distance
    A = np.array([0.0, 0.0, 0.0]); B = np.array([1.0, 0.0, 0.0]); C = np.array([0.0, 1.0, 0.0])
    P = np.array([300.0, 200.0, 0.0])
    c = (A + B + C) / 3
    assert abs(_potential_in_plane(P, A, B, C) * np.linalg.norm(P - c) / 0.5 - 1) < 1e-5


# -------------------------------------------------------------- geometry --
def test_surface_curls_closed_form():
    V, F = inputs.icosphere(1)
    V = inputs.jitter(V, F, 0.05, 3)
    o = Oracle(V, F, inputs.equidistant_grid(5, 1.0), psi_mode="direct")
    for e in range(0, F.shape[0], 7):
        n, area, curl = o.tri_geom(e)
        P = V[F[e]]
        c = np.cross(P[1] - P[0], P[2] - P[0])
        assert abs(area - 0.5 * np.linalg.norm(c)) < 1e-15
        assert np.allclose(n, c / np.linalg.norm(c), atol=1e-15)
        assert np.dot(n, P.mean(axis=0)) > 0  # outward on the sphere
        for a in range(3):
            edge = P[(a + 2) % 3] - P[(a + 1) % 3]
            assert np.allclose(curl[a], -edge / (2 * area), atol=1e-13)  # n x grad = -e_a/(2T)
        assert np.allclose(curl.sum(axis=0), 0, atol=1e-13)


def test_triangle_distance_bounds():
    V, F = inputs.icosphere(2)
    V = inputs.jitter(V, F, 0.05, 1)
    o = Oracle(V, F, inputs.equidistant_grid(5, 1.0), psi_mode="direct")
    rng = np.random.default_rng(1)
    u = rng.dirichlet([1, 1, 1], size=1500)
    u = np.vstack([u, np.eye(3), [[0.5, 0.5, 0], [0, 0.5, 0.5], [0.5, 0, 0.5]]])
    for s, q in [(0, 5), (3, 100), (17, 18), (40, 41), (7, 300), (12, 12), (2, 250)]:
        dmin, dmax = o.tri_bounds(s, q)
        X = u @ V[F[s]]
        Y = u @ V[F[q]]
        D = np.linalg.norm(X[:, None] - Y[None], axis=2)
        assert dmax == pytest.approx(np.linalg.norm(V[F[s]][:, None] - V[F[q]][None], axis=2).max(), abs=1e-15)
        assert D.max() <= dmax + 1e-15
        assert dmin <= D.min() + 1e-15
        if len(set(F[s]) & set(F[q])):
            assert dmin == 0.0
        else:
            assert D.min() - dmin < 0.05 * (D.min() + 1e-3)
    # exact value for two parallel segments' triangles: a translated copy
    Vt = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 0.3], [1, 0, 0.3], [0, 1, 0.3]], float)
    Ft = np.array([[0, 1, 2], [3, 5, 4]], np.int32)
    ot = Oracle(Vt, Ft, inputs.equidistant_grid(5, 1.0), psi_mode="direct")
    dmin, dmax = ot.tri_bounds(0, 1)
    assert abs(dmin - 0.3) < 1e-15 and abs(dmax - math.sqrt(2 + 0.09)) < 1e-15
    # exact value attained only between edge interiors: the x-axis edge of a
    # triangle that drops steeply away (z = 10 y, y <= 0) and the crossing
    # edge x = 0, z = 0.3 of a vertical triangle above it; every vertex-face
    # foot point falls outside the other triangle, so dmin = 0.3 comes from
    # the segment-segment distance alone
    Ve = np.array([[-1, 0, 0], [1, 0, 0], [0, -0.1, -1], [0, -1, 0.3], [0, 1, 0.3], [0, 0, 1.3]], float)
    oe = Oracle(Ve, Ft, inputs.equidistant_grid(5, 1.0), psi_mode="direct")
    for s, q in [(0, 1), (1, 0)]:
        assert abs(oe.tri_bounds(s, q)[0] - 0.3) < 1e-15


# ------------------------------------------------------------ block list --
def _support(t, kb, ib):
    N = t.size
    tl = 0.0 if kb == 0 else t[kb - 1]
    tr_i = t[-1] if ib == N - 1 else t[ib + 1]
    tr_k = t[-1] if kb == N - 1 else t[kb + 1]
    tl_i = 0.0 if ib == 0 else t[ib - 1]
    return max(0.0, tl - tr_i), tr_k - tl_i


def test_unique_block_list_equidistant():
    V, F = inputs.icosphere(1)
    t = inputs.equidistant_grid(17, 4.0)
    o = Oracle(V, F, t, psi_mode="direct")
    diam = o.diam()
    N = t.size
    got = {(b[0], b[1]) for b in o.blocks()}
    want = set()
    for k in range(N):
        for i in range(N):
            if not (i in (0, 1) or k == N - 1 or (k, i) in ((1, 2), (N - 2, N - 1))):
                continue
            a, b = _support(t, k, i)
            if i <= k + 1 and b > a and a < diam - 1e-12 * t[-1]:
                want.add((k, i))
    assert got == want
    assert len(got) <= 3 * N  # Sec. 5.1: at most 3N blocks
    assert all(i <= k + 1 for k, i in got)  # block Hessenberg


@pytest.mark.parametrize("N,dt,diam", [(17, 0.25, 1.97), (65, 0.0625, 1.97), (129, 0.05, 1.97), (30, 0.1, 1.03), (12, 0.3, 1.4)])
def test_inner_block_count_closed_form(N, dt, diam):
    # n_z (Sec. 5.1) with the observed number of nonzero first-column blocks;
    # the paper's estimate of that number is an upper bound
    t = np.arange(N) * dt
    inner = col1 = 0
    for k in range(N):
        for i in range(min(k + 2, N)):
            a, b = _support(t, k, i)
            nz = b > a and a < diam
            inner += nz and 1 <= k <= N - 2 and 1 <= i <= N - 2
            col1 += nz and i == 0
    nz = 0.5 * (N * N - N - 4) - (N - col1 - 2) / 2 * max(N - col1 - 1, 0)
    assert nz == inner
    assert col1 <= min(N, math.ceil(2 * diam / dt) + 2)


def test_graded_blocks_are_all_nonzero_hessenberg():
    V, F = inputs.icosphere(0)
    t = inputs.graded_grid(10, 1.2, 3.0)
    o = Oracle(V, F, t, equidistant=False, psi_mode="direct")
    got = {(b[0], b[1]) for b in o.blocks()}
    N = t.size
    want = {(k, i) for k in range(N) for i in range(min(k + 2, N)) if _support(t, k, i)[0] < o.diam() - 1e-12 * t[-1]}
    assert got == want


# ------------------------------------------------------- assembled blocks --
def _dense(o, blks):
    res = o.assemble_rows(np.arange(o.M), np.asarray(blks))
    out = {}
    for b in blks:
        Af = np.zeros((o.M, o.M)); An = np.zeros((o.M, o.M))
        for l, (c, f, n) in enumerate(res[int(b)]):
            Af[l, c] = f; An[l, c] = n
        out[int(b)] = (Af, An)
    return out


def test_block_symmetry():
    # both terms of Eq. MatrixEntries are symmetric under x <-> y with (j,l)
    # swapped; the 7-point far rule keeps that exactly, Sauter-Schwab up to
    # its quadrature error
    V, F = inputs.icosphere(1)
    V = inputs.jitter(V, F, 0.03, 5)
    o = Oracle(V, F, inputs.equidistant_grid(9, 2.0), psi_mode="interp")
    blks = list(range(o.num_blocks()))
    D = _dense(o, blks)
    for b in blks:
        Af, An = D[b]
        nf = np.linalg.norm(Af)
        if nf > 0:
            assert np.linalg.norm(Af - Af.T) <= 1e-13 * nf
        nn = np.linalg.norm(An)
        if nn > 0:
            assert np.linalg.norm(An - An.T) <= 5e-2 * nn
        # the pattern is symmetric
        P = (Af != 0) | (An != 0)
        assert np.array_equal(P, P.T)


def test_pattern_matches_sampled_distances():
    # Eq. SparsitySmallBlock: entry (l,j) is structural iff the support of psi
    # meets [mindist_{l,j}, maxdist_{l,j}]; check against sampled stars
    V, F = inputs.tiny_meshes()["octa"]
    t = inputs.equidistant_grid(9, 1.6)
    o = Oracle(V, F, t, equidistant=False, psi_mode="direct")
    rng = np.random.default_rng(2)
    u = np.vstack([rng.dirichlet([1, 1, 1], size=400), np.eye(3)])
    stars = {v: np.vstack([u @ V[F[e]] for e in range(F.shape[0]) if v in F[e]]) for v in range(o.M)}
    lo = np.zeros((o.M, o.M)); hi = np.zeros((o.M, o.M))
    for l in range(o.M):
        for j in range(o.M):
            D = np.linalg.norm(stars[l][:, None] - stars[j][None], axis=2)
            lo[l, j], hi[l, j] = D.min(), D.max()
    res = o.assemble_rows(np.arange(o.M), np.arange(o.num_blocks()))
    for b, (kb, ib, m2, m1, a, bb) in enumerate(o.blocks()):
        for l, (c, f, n) in enumerate(res[b]):
            row = set(c.tolist())
            for j in range(o.M):
                if lo[l, j] < bb - 1e-3 and hi[l, j] > a + 1e-3:
                    assert j in row
                if lo[l, j] > bb + 0.05 or hi[l, j] < a - 1e-9:
                    assert j not in row


def test_pattern_counts_on_fine_grid():
    # the same criterion with supports (4 dt = 0.16) narrow against the
    # distance range of the stars [0, 1]: every row length lies between the
    # number of columns that certainly qualify (sampled star distances inside
    # the support by a margin; the sampled maximum is exact, since it sits at
    # vertices, the sampled minimum is an upper bound) and the number that
    # possibly qualify
    V, F = inputs.tiny_meshes()["icosa"]
    t = inputs.equidistant_grid(41, 1.6)
    o = Oracle(V, F, t, equidistant=False, psi_mode="direct")
    rng = np.random.default_rng(3)
    u = np.vstack([rng.dirichlet([1, 1, 1], size=200), np.eye(3)])
    stars = {v: np.vstack([u @ V[F[e]] for e in range(F.shape[0]) if v in F[e]]) for v in range(o.M)}
    lo = np.zeros((o.M, o.M)); hi = np.zeros((o.M, o.M))
    for l in range(o.M):
        for j in range(o.M):
            D = np.linalg.norm(stars[l][:, None] - stars[j][None], axis=2)
            lo[l, j], hi[l, j] = D.min(), D.max()
    err = 0.06  # sampling error of the minimum, well above what 200 points leave
    counts = o.pattern_counts(np.arange(o.M), np.arange(o.num_blocks()))
    for b, (kb, ib, m2, m1, a, bb) in enumerate(o.blocks()):
        sure = ((lo < bb - 1e-9) & (hi > a + 1e-9)).sum(axis=1)
        maybe = ((lo - err < bb) & (hi > a - 1e-9)).sum(axis=1)
        assert (sure <= counts[b]).all() and (counts[b] <= maybe).all(), (kb, ib)


def test_toeplitz_block_reuse():
    # Eq. relationAtildeBlock: inner blocks depend on k~ - i~ only
    V, F = inputs.icosphere(1)
    t = inputs.equidistant_grid(11, 2.5)
    o = Oracle(V, F, t, equidistant=False, psi_mode="interp")
    idx = {(b[0], b[1]): n for n, b in enumerate(o.blocks())}
    pairs = [((4, 2), (6, 4)), ((3, 3), (7, 7)), ((2, 3), (5, 6)), ((5, 1), (8, 4))]
    blks = sorted({idx[p] for pr in pairs for p in pr})
    D = _dense(o, blks)
    for p, q in pairs:
        A = sum(D[idx[p]]); B = sum(D[idx[q]])
        assert np.linalg.norm(A - B) <= 1e-12 * np.linalg.norm(A)
    # negative control: a graded grid loses it
    tg = inputs.graded_grid(10, 1.15, 2.5)
    og = Oracle(V, F, tg, equidistant=False, psi_mode="interp")
    idg = {(b[0], b[1]): n for n, b in enumerate(og.blocks())}
    Dg = _dense(og, [idg[(4, 2)], idg[(6, 4)]])
    A = sum(Dg[idg[(4, 2)]]); B = sum(Dg[idg[(6, 4)]])
    assert np.linalg.norm(A - B) > 1e-3 * np.linalg.norm(A)


def test_order_symmetry_of_inner_blocks():
    # Eq. relationAblock (p >= 1): for inner k~, i~ the block of test order
    # m2 and trial order m1 is (-1)^(m1+m2) times the block with the orders
    # swapped (from Eq. symmetryXi and Eq. symmetryXip); a first-column block
    # has no such relation (negative control)
    V, F = inputs.icosphere(1)
    t = inputs.equidistant_grid(9, 2.0)
    o = Oracle(V, F, t, p=2, equidistant=False, psi_mode="interp")
    idx = {b[:4]: n for n, b in enumerate(o.blocks())}
    cases = [((4, 3), 0, 1), ((4, 3), 1, 2), ((5, 2), 0, 2), ((3, 4), 0, 1)]
    blks = sorted({idx[(k, i, a, b)] for (k, i), a, b in cases} | {idx[(k, i, b, a)] for (k, i), a, b in cases}
                  | {idx[(4, 0, 0, 1)], idx[(4, 0, 1, 0)]})
    D = _dense(o, blks)
    for (k, i), a, b in cases:
        A = sum(D[idx[(k, i, a, b)]]); B = sum(D[idx[(k, i, b, a)]])
        assert np.linalg.norm(A) > 0
        assert np.linalg.norm(A - (-1) ** (a + b) * B) <= 1e-10 * np.linalg.norm(A), (k, i, a, b)
    A = sum(D[idx[(4, 0, 0, 1)]]); B = sum(D[idx[(4, 0, 1, 0)]])
    assert np.linalg.norm(A + B) > 1e-2 * np.linalg.norm(A)


def test_far_and_near_quadrature_convergence():
    V, F = inputs.tiny_meshes()["icosa"]
    o = Oracle(V, F, inputs.equidistant_grid(9, 2.0), equidistant=False, psi_mode="interp")
    blks = np.arange(o.num_blocks())
    # far pair: 7-point rule vs product Gauss rules
    s, q = 0, 12
    assert len(set(F[s]) & set(F[q])) == 0
    L7 = o.pair_local(s, q, blks)
    L12 = o.pair_local(s, q, blks, far_n=12)
    L20 = o.pair_local(s, q, blks, far_n=20)
    L30 = o.pair_local(s, q, blks, far_n=30)
    sc = np.abs(L30).max()
    e = [np.abs(L - L30).max() / sc for L in (L7, L12, L20)]
    assert e[0] > e[1] > e[2] and e[1] < 1e-5 and e[0] < 0.15
    # near pairs (coincident / edge / vertex): Sauter-Schwab orders 4..16
    for q in [0, 1, 3]:
        kase = len(set(F[s]) & set(F[q]))
        assert kase > 0
        ref = o.pair_local(s, q, blks, near_n=16)
        sc = np.abs(ref).max()
        e = [np.abs(o.pair_local(s, q, blks, near_n=n) - ref).max() / sc for n in (4, 8, 12)]
        assert e[0] > e[1] > e[2] and e[2] < 1e-3


def _sphere_forms(o, blk, a, b):
    # closed forms on the unit sphere (n_x = x, n_x.n_y = 1 - r^2/2,
    # dGamma_y = 2 pi r dr): with K = psi/(4 pi r) and K~ = psi~/(4 pi r)
    #   1^T A 1 = 2 pi int_0^2 (1 - r^2/2) psi dr
    #   z^T A z = (2 pi/3) int (1 - r^2/2)^2 psi dr + (4 pi/3) int (1 - r^2/2) psi~ dr
    x, w = gauss_legendre(48)
    e = np.linspace(a, min(b, 2.0), 25)
    r = (e[:-1, None] + (e[1:] - e[:-1])[:, None] * x[None]).ravel()
    ww = ((e[1:] - e[:-1])[:, None] * w[None]).ravel()
    ps = o.psi_block(blk, r)
    c = 1 - r * r / 2
    one = 2 * np.pi * np.sum(ww * c * ps[:, 0])
    zz = 2 * np.pi / 3 * np.sum(ww * c * c * ps[:, 0]) + 4 * np.pi / 3 * np.sum(ww * c * ps[:, 1])
    return one, zz


@pytest.mark.slow
@pytest.mark.parametrize("p,keys,bound", [(0, [(1, 1, 0, 0), (2, 1, 0, 0)], 0.06),
                                          (1, [(2, 1, 0, 1), (2, 1, 1, 0), (2, 1, 1, 1)], 0.08)])
def test_sphere_bilinear_forms_converge(p, keys, bound):
    # p = 1 runs the same spatial assembly with the Legendre orders m2, m1;
    # the flat-triangle error falls by 4 to 10 per refinement (the pin), the
    # absolute bound only guards the level-2 size (0.072 for the p = 1
    # curl form of block (2, 1, 1, 1), 0.011 one level finer)
    t = inputs.equidistant_grid(5, 2.0)
    errs = {}
    for level in (1, 2):
        V, F = inputs.icosphere(level)
        o = Oracle(V, F, t, p=p, psi_mode="interp")
        idx = {b[:4]: n for n, b in enumerate(o.blocks())}
        sel = [idx[k] for k in keys]
        D = _dense(o, sel)
        z = V[:, 2]
        for n, blk in enumerate(sel):
            A = sum(D[blk])
            kb, ib, _, _, a, b = o.blocks()[blk]
            one, zz = _sphere_forms(o, blk, a, b)
            errs[(level, n)] = (abs(A.sum() - one) / abs(one), abs(z @ A @ z - zz) / abs(zz))
    for n in range(len(keys)):
        for f in range(2):
            assert errs[(2, n)][f] < 0.4 * errs[(1, n)][f]
            assert errs[(2, n)][f] < bound
