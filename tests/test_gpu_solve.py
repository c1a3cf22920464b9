"""GPU right-hand side and block-Hessenberg solve through the C ABI against
the oracle (the 320-triangle sphere, 16 steps of 0.25 on [0, 4], plane-wave
Neumann datum d = (0, 0, 1), pulse centre 1.0 after first contact, width 0.2).

* RHS: the CUDA g_k(l) against the oracle's for every kind, 1e-11 relative.
* Solve: restarted GMRES(50) to 1e-10 on the FP64 path against the oracle's
  dense LU solution of its own FP64 matrix; the true residual of the GPU
  solution against the oracle's block-Hessenberg product. The mixed path's
  product rounds x and its products to FP32 (relative noise ~1e-7), so its
  solve is asked for 1e-6.
"""
import numpy as np
import pytest

from paper_1503_07221_gb300 import inputs

pytestmark = pytest.mark.gpu

# u_inc = f(t - x.d - c0): c0 = 1.0 + 1 puts the pulse centre 1.0 after the
# wave first touches the unit sphere (x.d = -1)
PLANE = (0.0, 0.0, 1.0, 2.0, 0.2)


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
def case():
    V, F = inputs.icosphere(2)
    t = inputs.equidistant_grid(17, 4.0)
    return V, F, t


@pytest.fixture(scope="module")
def orc(case):
    from oracle.oracle import Oracle
    V, F, t = case
    return Oracle(V, F, t, psi_mode="interp")


@pytest.mark.parametrize("kind,params", [(0, PLANE), (1, ()), (2, ())])
def test_rhs_matches_oracle(td, case, orc, kind, params):
    V, F, t = case
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=0)
    g = asm.rhs(kind, params).cpu().numpy()
    ref = orc.rhs(kind, params)
    err = np.abs(g - ref).max() / np.abs(ref).max()
    print("rhs kind %d: max rel %.3e" % (kind, err))
    assert err < 1e-11


def test_solve_fp64_matches_dense_lu(td, case, orc):
    import torch
    V, F, t = case
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=0)
    asm.assemble()
    g = asm.rhs(0, PLANE)
    # tolerance 1e-12: with the measured condition (error / residual ~ 1e2)
    # the iterate then meets the 1e-8 agreement with the dense LU solution
    alpha, it, rr = asm.solve(g, restart=50, tol=1e-12, max_iter=6000)
    alpha2, it2, rr2 = asm.solve(g, restart=50, tol=1e-12, max_iter=6000)
    torch.cuda.synchronize()
    a = alpha.cpu().numpy()
    assert np.array_equal(a, alpha2.cpu().numpy()) and it == it2, "solve is not deterministic"
    ref = orc.solve_dense(orc.rhs(0, PLANE))
    err = np.linalg.norm(a - ref) / np.linalg.norm(ref)
    res = np.linalg.norm(orc.hessenberg_apply(a) - orc.rhs(0, PLANE)) / np.linalg.norm(orc.rhs(0, PLANE))
    print("GMRES(50) fp64: %d iterations, rel res %.3e, vs dense LU %.3e, true residual %.3e" % (it, rr, err, res))
    assert rr <= 1e-12
    assert res <= 1e-11
    assert err <= 1e-8


def test_solve_mixed_converges(td, case):
    import torch
    V, F, t = case
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=1)
    asm.assemble()
    g = asm.rhs(0, PLANE)
    alpha, it, rr = asm.solve(g, restart=50, tol=1e-6)
    r = asm.hessenberg_apply(alpha) - g
    torch.cuda.synchronize()
    res = float(torch.linalg.norm(r) / torch.linalg.norm(g))
    print("GMRES(50) mixed: %d iterations, rel res %.3e (recomputed %.3e)" % (it, rr, res))
    assert rr <= 1e-6 and res <= 2e-6


def test_solve_errors(td, case):
    V, F, t = case
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=1)
    g = asm.rhs(1)
    with pytest.raises(td.TdbemError) as e:
        asm.solve(g)
    assert e.value.code == td.E_NOT_ASSEMBLED
    asm.assemble()
    with pytest.raises(td.TdbemError) as e:
        asm.solve(g, restart=0)
    assert e.value.code == td.E_INVALID_ARG
    with pytest.raises(td.TdbemError) as e:
        asm.rhs(0, (0.0, 0.0, 0.0, 1.0, 0.2))
    assert e.value.code == td.E_INVALID_ARG
    with pytest.raises(td.TdbemError) as e:
        asm.rhs(7)
    assert e.value.code == td.E_INVALID_ARG
