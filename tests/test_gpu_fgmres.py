"""GPU flexible GMRES with the recursive block-Hessenberg preconditioner
(Sec. 4.2, Algorithm 1) through the C ABI against the oracle
(oracle/krylov.py) on the oracle's own FP64 matrix.

Case: the 320-triangle sphere (the mesh of the solver experiments of
Sec. 6), equidistant grids on [0, 6], the n = 0 sphere datum of Sec. 6.1.

* One preconditioner application, FP64 path, inner tolerance 1e-30 (every
  inner cycle runs its full step count, so both sides take the same path):
  relative difference 1e-9. Both sides solve the same small least-squares
  problems; the matrices differ by ~1e-13 relative.
* Whole solves at the experiments' tolerance 1e-5: the same outer iteration
  count as the oracle (+-1: a step whose estimate lands within rounding of
  the threshold may fall either way), true residual <= 1e-5, and the dense
  solution within the residual times a conditioning allowance.
* Degenerate splittings: N = 5 (the smallest grid the assembler takes),
  ragged halves 3 + 2, then 2 + 1 and 1 + 1, and more levels than halvings
  (the extra levels meet one-block ranges and leave them unpreconditioned).
  At N = 5 (dt = 1.5) the inner diagonal blocks have condition numbers near
  1e6 against 1e2 for the whole matrix, and the multi-level solves stall
  (the oracle's too, Sec. 6's "---" for N = 5): whole solves there are
  compared at one level only.
"""
import numpy as np
import pytest

from paper_1503_07221_gb300 import inputs

pytestmark = pytest.mark.gpu

T_END = 6.0


@pytest.fixture(scope="module")
def td():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1503_07221_gb300 import build, tdbem
    build.build()
    torch.cuda.set_device(0)
    tdbem.use_torch_allocator()
    return tdbem


@pytest.fixture(scope="module")
def sphere():
    return inputs.icosphere(2)


_cache = {}


def _case(td, sphere, N, precision=0):
    """(assembler, oracle dense matrix, oracle rhs) for N grid points."""
    import torch
    key = (N, precision)
    if key not in _cache:
        from oracle.oracle import Oracle
        V, F = sphere
        t = inputs.equidistant_grid(N, T_END)
        asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=precision)
        asm.assemble()
        if ("o", N) not in _cache:
            o = Oracle(V, F, t, psi_mode="interp")
            _cache[("o", N)] = (o.full_matrix(), o.rhs(1).ravel(), o.M)
        _cache[key] = asm
    A, g, M = _cache[("o", N)]
    return _cache[key], A, g, M


@pytest.mark.parametrize("N,inner", [(11, (10,)), (11, (5,)), (11, (2, 10)), (11, (3, 3, 3)),
                                     (5, (4, 4, 4, 4)), (5, (6,))])
def test_preconditioner_matches_oracle(td, sphere, N, inner):
    import torch
    from oracle.krylov import RecursivePreconditioner
    asm, A, g, M = _case(td, sphere, N)
    r = np.random.default_rng(7).standard_normal(N * M)
    z = asm.precondition(torch.from_numpy(r).cuda(), inner=inner, tol=1e-30).cpu().numpy()
    ref = RecursivePreconditioner(A, N, M, inner, 1e-30).apply(r)
    err = np.linalg.norm(z - ref) / np.linalg.norm(ref)
    print("M^-1 r, N=%d inner=%s: rel diff %.3e" % (N, inner, err))
    assert err <= 1e-9


@pytest.mark.parametrize("N,inner", [(11, ()), (11, (10,)), (11, (5,)), (11, (2, 10)), (6, (10,)), (5, (10,))])
def test_fgmres_matches_oracle(td, sphere, N, inner):
    import torch
    from oracle.krylov import solve
    asm, A, g, M = _case(td, sphere, N)
    tol = 1e-5
    x_ref, it_ref, hist = solve(A, N, M, g, 50, tol, 5000, inner)
    gd = torch.from_numpy(g).cuda()
    alpha, it, rr = asm.solve_fgmres(gd, restart=50, tol=tol, max_iter=5000, inner=inner)
    a = alpha.cpu().numpy()
    true_rr = np.linalg.norm(A @ a - g) / np.linalg.norm(g)
    ref = np.linalg.solve(A, g)
    err = np.linalg.norm(a - ref) / np.linalg.norm(ref)
    print("FGMRES(50,%s) N=%d: %d iterations (oracle %d), rel res %.3e (oracle matrix %.3e), vs LU %.3e"
          % (inner, N, it, it_ref, rr, true_rr, err))
    assert abs(it - it_ref) <= 1
    assert rr <= tol and true_rr <= 1.01 * tol
    assert err <= 1e3 * tol


def test_max_iter_bounds_a_stalled_solve(td, sphere):
    # FGMRES(50, 2(2, 10)) on N = 6 stalls near 1e-2 (the oracle too). Where
    # a stalled flexible iteration with inexact inner solves stops depends on
    # rounding: multiplying every entry of the oracle's own matrix by
    # (1 + 1e-16 N(0, 1)) moves its final residual by 6-15 %. So the test
    # asks for the stall (the cap reached, the residual far above the
    # tolerance) at the oracle's level within a factor of 2.
    import torch
    from oracle.krylov import solve
    asm, A, g, M = _case(td, sphere, 6)
    _, it_ref, hist = solve(A, 6, M, g, 50, 1e-5, 120, (2, 10))
    alpha, it, rr = asm.solve_fgmres(torch.from_numpy(g).cuda(), restart=50, tol=1e-5, max_iter=120, inner=(2, 10))
    print("stalled: %d iterations, rel res %.3e (oracle %d, %.3e)" % (it, rr, it_ref, hist[-1]))
    assert it == it_ref == 120
    assert rr > 1e-3 and 0.5 * hist[-1] <= rr <= 2.0 * hist[-1]


def test_fgmres_deterministic_and_zero_rhs(td, sphere):
    import torch
    asm, A, g, M = _case(td, sphere, 11)
    gd = torch.from_numpy(g).cuda()
    a1, i1, r1 = asm.solve_fgmres(gd, inner=(2, 10))
    a2, i2, r2 = asm.solve_fgmres(gd, inner=(2, 10))
    assert i1 == i2 and r1 == r2 and torch.equal(a1, a2)
    z, iz, rz = asm.solve_fgmres(torch.zeros_like(gd), inner=(10,))
    assert iz == 0 and rz == 0.0 and not z.any()


def test_fgmres_mixed_precision_converges(td, sphere):
    import torch
    asm, A, g, M = _case(td, sphere, 11, precision=1)
    alpha, it, rr = asm.solve_fgmres(torch.from_numpy(g).cuda(), tol=1e-5, inner=(10,))
    true_rr = np.linalg.norm(A @ alpha.cpu().numpy() - g) / np.linalg.norm(g)
    print("mixed FGMRES(50,1(10)): %d iterations, rel res %.3e (oracle matrix %.3e)" % (it, rr, true_rr))
    assert rr <= 1e-5 and true_rr <= 2e-5


def test_fgmres_errors(td, sphere):
    import torch
    asm, A, g, M = _case(td, sphere, 11)
    gd = torch.from_numpy(g).cuda()
    for kw in (dict(restart=0), dict(restart=63), dict(tol=0.0), dict(tol=1.0), dict(max_iter=0),
               dict(inner=(0,)), dict(inner=(63,)), dict(inner=(2,) * 25)):
        with pytest.raises(td.TdbemError) as e:
            asm.solve_fgmres(gd, **kw)
        assert e.value.code == td.E_INVALID_ARG, kw
    with pytest.raises(td.TdbemError) as e:
        asm.precondition(gd, inner=())
    assert e.value.code == td.E_INVALID_ARG
    with pytest.raises(td.TdbemError) as e:
        asm.precondition(gd, inner=(10,), out=gd)
    assert e.value.code == td.E_INVALID_ARG
    V, F = sphere
    fresh = td.Assembler(td.Mesh(V, F), td.TimeGrid(inputs.equidistant_grid(11, T_END)), precision=0)
    with pytest.raises(td.TdbemError) as e:
        fresh.solve_fgmres(gd)
    assert e.value.code == td.E_NOT_ASSEMBLED
