"""Pins of the oracle's solver (oracle/krylov.py): flexible GMRES and the
recursive block-Hessenberg preconditioner of Sec. 4.2 (Algorithm 1).

* GMRES is the minimal-residual method on the Krylov space: after k steps
  from zero the iterate minimises |b - A x| over span{b, A b, ..., A^k-1 b}
  (brute force: QR of the explicit Krylov matrix and a least-squares solve).
* With a fixed preconditioner P the flexible method is right-preconditioned
  GMRES: x = P^-1 u with u minimal over the Krylov space of A P^-1.
* With exact inner solves the recursive preconditioner is the inverse of the
  block lower-triangular M that drops block (h - 1, h), h = ceil(N/2)
  (dense solve), at any number of levels.
* Woodbury structure (Sec. 4.2): A M^-1 - I has rank at most one block.
* The restarted solve reaches the dense solution of the assembled
  space-time system, preconditioned or not.
* Deflation (Sec. 4.1): M^-1 = I + U (|lam| T^-1 - I) U^T inverts
  M = I + U (T/|lam| - I) U^T, and with U an exact invariant subspace of the
  r smallest eigenvalues the spectrum of A M^-1 is lam_{r+1}, ..., lam_n
  and |lam_n| (r times); DGMRES(m, 0) is GMRES(m), and DGMRES(m, l)
  converges where GMRES(m) stalls.
"""
import numpy as np
import pytest

from oracle.krylov import RecursivePreconditioner, deflation_inverse, dgmres, fgmres, solve


def _rand_hessenberg(nblk, bs, seed, shift=4.0):
    """Random block-Hessenberg matrix (zero above the first block
    superdiagonal), diagonally shifted so every leading block is invertible."""
    rng = np.random.default_rng(seed)
    n = nblk * bs
    A = rng.standard_normal((n, n)) / np.sqrt(bs)
    for k in range(nblk):
        A[k * bs:(k + 1) * bs, (k + 2) * bs:] = 0.0
    return A + shift * np.eye(n)


def _krylov_min(A, b, k, Pinv=None):
    B = A if Pinv is None else A @ Pinv
    K = np.zeros((b.size, k))
    v = b.copy()
    for j in range(k):
        K[:, j] = v
        v = B @ v
    Q = np.linalg.qr(K)[0]
    u = Q @ np.linalg.lstsq(B @ Q, b, rcond=None)[0]
    return u if Pinv is None else Pinv @ u


def test_gmres_iterate_is_krylov_minimal_residual():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 40)) + 6.0 * np.eye(40)
    b = rng.standard_normal(40)
    for k in range(1, 11):
        x, it, _ = fgmres(lambda v: A @ v, b, k, 0.0, k)
        assert it == k
        ref = _krylov_min(A, b, k)
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref), k


def test_fixed_preconditioner_is_right_preconditioned_gmres():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((36, 36)) + 5.0 * np.eye(36)
    b = rng.standard_normal(36)
    P = np.tril(A)
    Pinv = np.linalg.inv(P)
    for k in (1, 3, 6, 9):
        x, _, _ = fgmres(lambda v: A @ v, b, k, 0.0, k, prec=lambda v: np.linalg.solve(P, v))
        ref = _krylov_min(A, b, k, Pinv)
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref), k


def test_estimate_is_true_residual_and_restart_converges():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((60, 60)) + 7.0 * np.eye(60)
    b = rng.standard_normal(60)
    x, it, hist = fgmres(lambda v: A @ v, b, 5, 1e-10, 500)
    assert hist[-1] <= 1e-10 and it > 5
    assert np.linalg.norm(b - A @ x) <= 1.01e-10 * np.linalg.norm(b)
    # the estimate of one step equals the true residual of the iterate
    xs, _, h1 = fgmres(lambda v: A @ v, b, 4, 0.0, 4)
    assert abs(h1[-1] - np.linalg.norm(b - A @ xs) / np.linalg.norm(b)) <= 1e-12
    # zero right-hand side: zero solution, no iteration
    x0, it0, _ = fgmres(lambda v: A @ v, np.zeros(60), 5, 1e-10, 50)
    assert it0 == 0 and not x0.any()


@pytest.mark.parametrize("nblk", [2, 5, 6, 7])
@pytest.mark.parametrize("levels", [1, 2, 3])
def test_exact_inner_solves_invert_block_triangular_M(nblk, levels):
    bs = 4
    A = _rand_hessenberg(nblk, bs, seed=10 + nblk)
    h = (nblk + 1) // 2
    M = A.copy()
    M[(h - 1) * bs:h * bs, h * bs:(h + 1) * bs] = 0.0
    assert np.abs(A - M).max() > 0.1  # the dropped block is really there
    n = nblk * bs
    P = RecursivePreconditioner(A, nblk, bs, inner=(n,) * levels, tol=1e-15)
    r = np.random.default_rng(5).standard_normal(n)
    z = P.apply(r)
    ref = np.linalg.solve(M, r)
    assert np.linalg.norm(z - ref) <= 1e-9 * np.linalg.norm(ref)


def test_preconditioned_operator_is_rank_one_block_from_identity():
    nblk, bs = 6, 4
    n = nblk * bs
    A = _rand_hessenberg(nblk, bs, seed=21)
    P = RecursivePreconditioner(A, nblk, bs, inner=(n,), tol=1e-15)
    Minv = np.stack([P.apply(e) for e in np.eye(n)], axis=1)
    s = np.linalg.svd(A @ Minv - np.eye(n), compute_uv=False)
    assert s[bs - 1] > 1e-3 and s[bs] <= 1e-9 * s[0]


def test_inexact_inner_solves_are_the_stated_iteration_counts():
    # one level, i_1 = 1: each half solve is one minimal-residual step, so
    # y1 = (r1.(A11 r1) / |A11 r1|^2) r1
    nblk, bs = 4, 3
    A = _rand_hessenberg(nblk, bs, seed=31)
    P = RecursivePreconditioner(A, nblk, bs, inner=(1,), tol=1e-15)
    r = np.random.default_rng(6).standard_normal(nblk * bs)
    z = P.apply(r)
    n1 = 2 * bs
    A11, A21, A22 = A[:n1, :n1], A[n1:, :n1], A[n1:, n1:]
    q = A11 @ r[:n1]
    y1 = (r[:n1] @ q) / (q @ q) * r[:n1]
    t = r[n1:] - A21 @ y1
    q2 = A22 @ t
    y2 = (t @ q2) / (q2 @ q2) * t
    assert np.allclose(z, np.concatenate([y1, y2]), rtol=1e-12, atol=1e-14)


@pytest.fixture(scope="module")
def system():
    from oracle.oracle import Oracle
    from paper_1503_07221_gb300 import inputs
    V, F = inputs.icosphere(1)
    o = Oracle(V, F, inputs.equidistant_grid(9, 3.0))
    return o.full_matrix(), o.N, o.M, o.rhs(1).ravel()


@pytest.mark.parametrize("inner", [(), (10,), (5,), (2, 10)])
def test_solve_reaches_dense_solution(system, inner):
    A, N, M, g = system
    x, it, hist = solve(A, N, M, g, 50, 1e-10, 3000, inner)
    ref = np.linalg.solve(A, g)
    assert hist[-1] <= 1e-10
    assert np.linalg.norm(A @ x - g) <= 1.5e-10 * np.linalg.norm(g)
    assert np.linalg.norm(x - ref) <= 1e-6 * np.linalg.norm(ref), (inner, it)


def _small_eigen_matrix(n=80, seed=0):
    """Q R Q^T with Q orthogonal, R upper triangular: eigenvalues the
    diagonal, four of modulus <= 0.05 and the rest in [1, 10]."""
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    d = np.concatenate([[1e-2, 2e-2, -3e-2, 5e-2], rng.uniform(1.0, 10.0, n - 4)])
    R = np.diag(d) + np.triu(rng.standard_normal((n, n)) * 0.05, 1)
    return Q @ R @ Q.T, d


def test_deflation_preconditioner_claims():
    import scipy.linalg as sla
    A, d = _small_eigen_matrix()
    n = A.shape[0]
    _, S, r = sla.schur(A, output="real", sort=lambda re, im: np.hypot(re, im) < 0.1)
    assert r == 4
    U = S[:, :r]
    lam = np.abs(d).max()
    Minv, T = deflation_inverse(lambda v: A @ v, U, lam)
    Mi = np.column_stack([Minv(e) for e in np.eye(n)])
    M = np.eye(n) + U @ (T / lam - np.eye(r)) @ U.T
    assert np.abs(M @ Mi - np.eye(n)).max() < 1e-11
    ev = np.sort_complex(np.linalg.eigvals(A @ Mi))
    want = np.sort_complex(np.concatenate([d[4:], [lam] * r]).astype(complex))
    assert np.abs(ev - want).max() < 1e-5


def test_dgmres_without_deflation_is_gmres():
    A, _ = _small_eigen_matrix(seed=2)
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    x1, it1, h1 = fgmres(lambda v: A @ v, b, 10, 1e-10, 120)
    x2, it2, h2, U = dgmres(lambda v: A @ v, b, 10, 0, 8, 1e-10, 120)
    assert it1 == it2 and np.array_equal(x1, x2) and U.shape[1] == 0


def test_dgmres_restores_convergence():
    A, _ = _small_eigen_matrix()
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    x0, it0, _ = fgmres(lambda v: A @ v, b, 10, 1e-10, 600)
    assert np.linalg.norm(b - A @ x0) > 1e-2 * np.linalg.norm(b)  # GMRES(10) stalls
    x, it, _, U = dgmres(lambda v: A @ v, b, 10, 2, 8, 1e-10, 600)
    assert it < 200 and U.shape[1] == 8
    assert np.linalg.norm(b - A @ x) <= 1e-9 * np.linalg.norm(b)
