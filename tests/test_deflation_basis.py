"""Host routine of DGMRES(m, l) (Sec. 4.1) through the C ABI, no device:
tdbem_deflation_basis against scipy's real Schur decomposition sorted by
eigenvalue modulus, as the oracle's DGMRES takes it.

For random upper Hessenberg matrices (real spectra, complex pairs, a
cluster near zero) and several l: the dimension equals scipy's sdim (a
complex pair counts twice), the basis is orthonormal, it spans the same
subspace as scipy's leading Schur vectors (projectors within 1e-8), the
subspace is invariant (||H B - B (B^T H B)|| <= 1e-10 ||H||), and the
largest modulus equals that of numpy's eigenvalues.
"""
import numpy as np
import pytest


def _lib():
    from paper_1503_07221_gb300 import tdbem
    try:
        tdbem.lib()
    except (RuntimeError, OSError) as e:
        pytest.skip("libtdbem not built: %s" % e)
    return tdbem


def _hessenberg(m, seed, kind):
    import scipy.linalg as sla
    rng = np.random.default_rng(seed)
    if kind == "random":
        A = rng.standard_normal((m, m))
    elif kind == "cluster":
        # a few eigenvalues near zero, the rest of modulus ~1, non-normal
        d = np.concatenate([rng.uniform(1e-3, 1e-2, 4), rng.uniform(0.5, 1.5, m - 4)])
        Q = np.linalg.qr(rng.standard_normal((m, m)))[0]
        A = Q @ (np.diag(d) + 0.1 * np.triu(rng.standard_normal((m, m)), 1)) @ Q.T
    else:  # rotations: complex pairs of distinct moduli
        blocks = []
        for k in range(m // 2):
            r, th = 0.2 + k, 0.3 + 0.1 * k
            blocks.append(r * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]]))
        D = sla.block_diag(*blocks)
        if m % 2:
            D = sla.block_diag(D, [[7.0]])
        Q = np.linalg.qr(rng.standard_normal((m, m)))[0]
        A = Q @ D @ Q.T
    H, _ = sla.hessenberg(A, calc_q=True)
    return np.triu(H, -1)


def _reference(H, l):
    import scipy.linalg as sla
    ev = np.linalg.eigvals(H)
    cut = np.sort(np.abs(ev))[min(l, H.shape[0]) - 1]
    _, S, sdim = sla.schur(H, output="real", sort=lambda re, im: np.hypot(re, im) <= cut * (1 + 1e-12))
    return S[:, :sdim], float(np.abs(ev).max())


@pytest.mark.parametrize("m,seed,kind", [(10, 0, "random"), (20, 1, "random"), (30, 2, "cluster"),
                                         (24, 3, "pairs"), (31, 4, "pairs"), (62, 5, "random")])
@pytest.mark.parametrize("l", [1, 2, 5])
def test_basis_matches_sorted_real_schur(m, seed, kind, l):
    td = _lib()
    H = _hessenberg(m, seed, kind)
    B, lm = td.deflation_basis(H, l)
    S, lref = _reference(H, l)
    assert B.shape[1] == S.shape[1]
    assert abs(lm - lref) <= 1e-12 * lref
    k = B.shape[1]
    assert np.abs(B.T @ B - np.eye(k)).max() < 1e-12
    assert np.abs(B @ B.T - S @ S.T).max() < 1e-8
    R = H @ B - B @ (B.T @ H @ B)
    assert np.linalg.norm(R) <= 1e-10 * np.linalg.norm(H)


def test_l_zero_gives_lam_max_only():
    td = _lib()
    H = _hessenberg(12, 7, "random")
    B, lm = td.deflation_basis(H, 0)
    assert B.shape[1] == 0
    assert abs(lm - np.abs(np.linalg.eigvals(H)).max()) <= 1e-12 * lm


def test_arguments():
    td = _lib()
    with pytest.raises(td.TdbemError) as e:
        td.deflation_basis(np.zeros((63, 63)), 1)
    assert e.value.code == td.E_INVALID_ARG
    with pytest.raises(td.TdbemError) as e:
        td.deflation_basis(np.eye(4), -1)
    assert e.value.code == td.E_INVALID_ARG
