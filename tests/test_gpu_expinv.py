"""The second smooth step of the time basis (basis_kind 1, built from
exp(-1/s)) through the C ABI, against the FP64 oracle with the same step:
identical block list and patterns, relative Frobenius error per block (FP64
1e-10, mixed 1e-6) on the 80-triangle sphere (9 points) and the workload of
the plain method (320 triangles, 17 points on [0, 4]); the right-hand side
of the same basis, and the graded path."""
import numpy as np
import pytest

from paper_1503_07221_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-6}


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


def _worst(td, V, F, t, precision, equidistant=True):
    from oracle.oracle import Oracle
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t, basis_kind=1), precision=precision)
    asm.assemble()
    orc = Oracle(V, F, t, psi_mode="interp", equidistant=equidistant, basis_kind=1)
    ob = orc.blocks()
    assert [(b[0], b[1]) for b in ob] == asm.blocks()
    M = V.shape[0]
    res = orc.assemble_rows(np.arange(M), np.arange(len(ob)))
    worst = 0.0
    for b in range(len(ob)):
        A = np.zeros((M, M))
        for which in (td.FAR, td.NEAR):
            rp, col, val = asm.block_csr_host(b, which)
            for l in range(M):
                A[l, col[rp[l]:rp[l + 1]]] += val[rp[l]:rp[l + 1]].astype(np.float64)
            if which == td.FAR:
                pat = (rp, col)
        R = np.zeros((M, M))
        for l, (c, f, n) in enumerate(res[b]):
            R[l, c] = f + n
            assert np.array_equal(c, pat[1][pat[0][l]:pat[0][l + 1]]), "pattern of block %d row %d" % (b, l)
        nr = np.linalg.norm(R)
        if nr > 0:
            worst = max(worst, np.linalg.norm(A - R) / nr)
    return asm, worst


@pytest.mark.parametrize("precision", [0, 1])
def test_expinv_sphere80(td, precision):
    V, F = inputs.icosphere(1)
    _, w = _worst(td, V, F, inputs.equidistant_grid(9, 2.0), precision)
    print("exp(-1/s) basis, 80 triangles, prec %d: worst block %.3e" % (precision, w))
    assert w < TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_expinv_sphere320_n17(td, precision):
    V, F = inputs.icosphere(2)
    _, w = _worst(td, V, F, inputs.equidistant_grid(17, 4.0), precision)
    print("exp(-1/s) basis, 320 triangles, prec %d: worst block %.3e" % (precision, w))
    assert w < TOL[precision]


def test_expinv_graded(td):
    V, F = inputs.icosphere(1)
    _, w = _worst(td, V, F, inputs.graded_grid(8, 1.25, 2.0), 0, equidistant=False)
    assert w < TOL[0]


def test_expinv_rhs(td):
    import torch
    from oracle.oracle import Oracle
    V, F = inputs.icosphere(2)
    t = inputs.equidistant_grid(17, 4.0)
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t, basis_kind=1))
    g = asm.rhs(td.RHS_SPHERE_N0).cpu().numpy()
    ref = Oracle(V, F, t, basis_kind=1).rhs(1, nt=32)  # 16 points per panel leave 4.5e-10 with this steeper step
    assert np.abs(g - ref).max() <= 1e-10 * np.abs(ref).max()
