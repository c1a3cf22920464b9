"""Pins of the oracle's block-Hessenberg matvec (Eq. Apartitioned, Sec. 5.1).

The reduced form looks every block up among the listed blocks of the
equidistant grid through Eq. relationAtildeBlock; it is pinned against the
same product built from every nonzero block assembled directly from its own
psi_{k,i} (no reuse), and the block structure against the support statement
of Sec. 5.1 (psi_{k,i} vanishes for t_k <= t_{i-2}).
"""
import numpy as np

from oracle.oracle import Oracle
from paper_1503_07221_gb300 import inputs


def _x(N, M, seed=0):
    return np.random.default_rng(seed).standard_normal((N, M))


def _pair(N, T):
    V, F = inputs.icosphere(1)
    t = inputs.equidistant_grid(N, T)
    return Oracle(V, F, t), Oracle(V, F, t, equidistant=False)


def test_reduced_matvec_equals_full_block_matrix():
    # N=9 on [0, 2]: no block is cut; N=17 on [0, 6.4]: dt = 0.4, the diam cut
    # removes the lags beyond diam = 2 (Sec. 5.1)
    for N, T in ((9, 2.0), (17, 6.4)):
        o, full = _pair(N, T)
        x = _x(N, o.M, seed=N)
        y = o.hessenberg_apply(x)
        z = full.hessenberg_apply(x)
        assert np.linalg.norm(y - z) <= 1e-12 * np.linalg.norm(z), (N, T)
        assert np.linalg.norm(z) > 0


def test_matvec_equals_dense_product():
    # the product loop against the dense space-time matrix laid out block by
    # block (row block k, column block i) from every directly assembled block
    _, full = _pair(9, 2.0)
    x = _x(full.N, full.M, seed=5)
    y = full.hessenberg_apply(x)
    z = (full.full_matrix() @ x.ravel()).reshape(full.N, full.M)
    assert np.linalg.norm(y - z) <= 1e-13 * np.linalg.norm(z)


def test_p1_reduced_matvec_and_dense_product():
    # p = 1: Eq. relationAtildeBlock holds for every pair of orders (m2, m1),
    # rows / columns k (p + 1) + m (Sec. 3 numbering); the product loop
    # against the dense matrix of the directly assembled blocks
    V, F = inputs.icosphere(0)
    t = inputs.equidistant_grid(8, 2.1)
    o = Oracle(V, F, t, p=1)
    full = Oracle(V, F, t, p=1, equidistant=False)
    x = _x(o.L, o.M, seed=11)
    y = o.hessenberg_apply(x)
    z = full.hessenberg_apply(x)
    d = (full.full_matrix() @ x.ravel()).reshape(full.L, full.M)
    assert y.shape == (16, 12) and np.linalg.norm(z) > 0
    assert np.linalg.norm(y - z) <= 1e-12 * np.linalg.norm(z)
    assert np.linalg.norm(z - d) <= 1e-13 * np.linalg.norm(d)
    # orders are not interchangeable: swapping m of x changes y
    xs = x.reshape(8, 2, 12)[:, ::-1].reshape(16, 12)
    assert not np.allclose(o.hessenberg_apply(xs), y)


def test_diam_cut_is_active_on_long_grid():
    o, full = _pair(17, 6.4)
    lags = {b[0] - b[1] for b in full.blocks()}
    assert max(lags) < 16  # some lower-left blocks are zero
    assert len(o.blocks()) < len(full.blocks())


def test_hessenberg_structure():
    # psi_{k,i} = 0 for t_k <= t_{i-2}: no nonzero block with i >= k + 2
    o, full = _pair(9, 2.0)
    assert all(b[1] <= b[0] + 1 for b in full.blocks())
    N = o.N
    assert all(o.block_source(k, i) is None for k in range(N) for i in range(k + 2, N))
    # the superdiagonal and the diagonal are present
    assert all(full.block_source(k, k + 1) is not None for k in range(N - 1))
    # y_k does not see x_i for i >= k + 2
    x = _x(N, o.M, seed=3)
    y = o.hessenberg_apply(x)
    x2 = x.copy()
    x2[5:] += 1.0
    y2 = o.hessenberg_apply(x2)
    assert np.array_equal(y[:3], y2[:3])
    assert not np.allclose(y[4:], y2[4:])


def test_rows_subset():
    o, _ = _pair(9, 2.0)
    x = _x(o.N, o.M, seed=5)
    y = o.hessenberg_apply(x)
    rows = np.array([0, 7, 41])
    ys = o.hessenberg_apply(x, rows=rows)
    assert np.allclose(ys[:, rows], y[:, rows], rtol=0, atol=1e-14 * np.abs(y).max())
    mask = np.ones(o.M, bool)
    mask[rows] = False
    assert not ys[:, mask].any()
