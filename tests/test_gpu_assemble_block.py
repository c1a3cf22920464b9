"""tdbem_assemble_block: one block (k, i) assembled on its own from its own
psi_{k,i}, read back through the C ABI with b = TDBEM_LAST_BLOCK.

* Against the FP64 oracle on the 80-triangle sphere (9 equidistant points):
  for a block of each kind (first column, inner, last row, superdiagonal,
  a special corner) the pattern is identical to the oracle's block that
  holds (k, i) and the values agree (relative Frobenius norm: FP64 1e-10,
  mixed 1e-6). For an inner block the oracle's holder is a different
  (k', i') (Eq. relationAtildeBlock): the GPU block built from psi_{k,i}
  reproduces it, a check of the Toeplitz reuse on the device.
* On a graded grid the single block equals the same block of the full
  assembly (same kernels, same panels): 1e-12.
* Arguments: i > k + 1, a zero block (support beyond diam) and reading the
  last block before any call are rejected with the documented codes.
"""
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


def _dense(M, asm, b, td):
    A = np.zeros((M, M))
    pats = []
    for which in (td.FAR, td.NEAR):
        rp, col, val = asm.block_csr_host(b, which)
        for l in range(M):
            A[l, col[rp[l]:rp[l + 1]]] += val[rp[l]:rp[l + 1]].astype(np.float64)
        pats.append((rp, col))
    return A, pats[0]


@pytest.mark.parametrize("precision", [0, 1])
def test_single_block_matches_oracle(td, precision):
    from oracle.oracle import Oracle
    V, F = inputs.icosphere(1)
    t = inputs.equidistant_grid(9, 2.0)
    M, N = V.shape[0], t.size
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=precision)
    orc = Oracle(V, F, t, psi_mode="interp")
    for k, i in ((3, 0), (5, 3), (6, 4), (N - 1, 2), (4, 5), (N - 1, N - 1), (N - 1, 0)):
        src = orc.block_source(k, i)
        if src is None:
            continue
        asm.assemble_block(k, i)
        info = asm.block_info(td.LAST_BLOCK)
        assert (info["k"], info["i"]) == (k, i)
        A, (rp, col) = _dense(M, asm, td.LAST_BLOCK, td)
        res = orc.assemble_rows(np.arange(M), [src])[src]
        R = np.zeros((M, M))
        for l, (c, f, n) in enumerate(res):
            R[l, c] = f + n
            assert np.array_equal(c, col[rp[l]:rp[l + 1]]), "pattern of block (%d, %d) row %d" % (k, i, l)
        err = np.linalg.norm(A - R) / np.linalg.norm(R)
        print("block (%d, %d) prec %d vs oracle block %s: %.3e" % (k, i, precision, orc.blocks()[src][:2], err))
        assert err < TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_single_block_equals_full_graded_assembly(td, precision):
    V, F = inputs.icosphere(1)
    t = inputs.graded_grid(8, 1.25, 2.0)
    M = V.shape[0]
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=precision)
    asm.assemble()
    blocks = asm.blocks()
    for b in (0, len(blocks) // 2, len(blocks) - 1):
        k, i = blocks[b]
        asm.assemble_block(k, i)
        A, _ = _dense(M, asm, td.LAST_BLOCK, td)
        R, _ = _dense(M, asm, b, td)
        assert np.linalg.norm(A - R) <= 1e-12 * np.linalg.norm(R), (k, i)


def test_single_block_rejects_bad_arguments(td):
    V, F = inputs.icosphere(1)
    t = inputs.equidistant_grid(33, 8.0)  # late blocks start beyond diam = 2
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=0)
    with pytest.raises(td.TdbemError) as e:
        asm.block_info(td.LAST_BLOCK)
    assert e.value.code == td.E_NOT_ASSEMBLED
    for k, i in ((3, 5), (30, 0), (40, 0)):
        with pytest.raises(td.TdbemError) as e:
            asm.assemble_block(k, i)
        assert e.value.code == td.E_INVALID_ARG
