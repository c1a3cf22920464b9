"""GPU parity on graded (non-equidistant) time grids: every nonzero block
(k, i), i <= k + 1, is its own unique block (no reuse along the diagonals),
assembled from its own psi_{k,i} with panels between the breakpoints
t_{k-a} - t_{i-b}. Checked against the FP64 oracle through the C ABI:
identical block list, identical pattern per block and row, relative
Frobenius error per block (FP64 path 1e-10, mixed path 1e-6), and the
block-Hessenberg product against the oracle's.
"""
import numpy as np
import pytest

from _pattern_fingerprint import device_fingerprint
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


def _dense(M, rp, col, val):
    A = np.zeros((M, M))
    for l in range(M):
        A[l, col[rp[l]:rp[l + 1]]] = val[rp[l]:rp[l + 1]]
    return A


def _compare(td, V, F, t, precision, rows=None, blocks=None):
    from oracle.oracle import Oracle
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=precision)
    asm.assemble()
    orc = Oracle(V, F, t, equidistant=False, psi_mode="interp")
    ob = orc.blocks()
    assert [(b[0], b[1]) for b in ob] == asm.blocks()
    M = V.shape[0]
    rows = np.arange(M) if rows is None else np.asarray(rows)
    blocks = np.arange(len(ob)) if blocks is None else np.asarray(blocks)
    res = orc.assemble_rows(rows, blocks)
    errs = []
    for b in blocks:
        b = int(b)
        rp, col, vf = asm.block_csr_host(b, td.FAR)
        rpn, coln, vn = asm.block_csr_host(b, td.NEAR)
        Af = _dense(M, rp, col, vf.astype(np.float64))[rows]
        An = _dense(M, rpn, coln, vn)[rows]
        R = np.zeros((rows.size, M))
        for r, (c, f, n) in enumerate(res[b]):
            l = rows[r]
            assert np.array_equal(c, col[rp[l]:rp[l + 1]]), "pattern of block %d row %d" % (b, l)
            R[r, c] = f + n
        nr = np.linalg.norm(R)
        e = np.linalg.norm(Af + An - R) / nr if nr > 0 else np.linalg.norm(Af + An)
        errs.append((e, b, ob[b][:2], nr))
    return asm, orc, errs


def _worst(errs):
    # relative error of every block whose norm is at least 1e-3 of the largest,
    # and every block's error against the largest block norm
    nmax = max(e[3] for e in errs)
    rel = max((e for e in errs if e[3] >= 1e-3 * nmax), key=lambda e: e[0])
    absmax = max(e[0] * e[3] for e in errs) / nmax
    return rel, absmax


@pytest.mark.parametrize("precision", [0, 1])
def test_graded_sphere80(td, precision):
    # strongly graded: 8 steps with ratio 1.25 on [0, 2]; uneven panels everywhere
    V, F = inputs.icosphere(1)
    t = inputs.graded_grid(8, 1.25, 2.0)
    _, _, errs = _compare(td, V, F, t, precision)
    rel, absmax = _worst(errs)
    print("graded sphere80 prec %d: worst rel %.3e at %s, abs %.3e" % (precision, rel[0], rel[2], absmax))
    assert rel[0] < TOL[precision], rel
    assert absmax < TOL[precision], absmax


@pytest.mark.parametrize("precision", [0, 1])
def test_graded_torus_small(td, precision):
    # torus R = 1, r = 0.4 on a 16 x 8 quad grid (256 triangles), 12 steps of
    # ratio 1.1 on [0, 3]: several tiles of 32 trial triangles and a ragged tail
    V, F = inputs.torus(1.0, 0.4, 16, 8)
    t = inputs.graded_grid(12, 1.1, 3.0)
    rows = np.arange(0, V.shape[0], 5)
    _, _, errs = _compare(td, V, F, t, precision, rows=rows)
    rel, absmax = _worst(errs)
    print("graded torus256 prec %d: worst rel %.3e at %s, abs %.3e" % (precision, rel[0], rel[2], absmax))
    assert rel[0] < TOL[precision], rel
    assert absmax < TOL[precision], absmax


@pytest.mark.parametrize("precision", [0, 1])
def test_graded_matvec(td, precision):
    import torch
    from oracle.oracle import Oracle
    V, F = inputs.icosphere(1)
    t = inputs.graded_grid(10, 1.2, 2.5)
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=precision)
    asm.assemble()
    orc = Oracle(V, F, t, equidistant=False, psi_mode="interp")
    x = np.random.default_rng(3).standard_normal((t.size, V.shape[0]))
    y = asm.hessenberg_apply(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = orc.hessenberg_apply(x)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    print("graded matvec prec %d: %.3e" % (precision, err))
    assert err < {0: 1e-12, 1: 1e-6}[precision]


def test_graded_deterministic(td):
    V, F = inputs.icosphere(1)
    t = inputs.graded_grid(8, 1.25, 2.0)
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=1)
    asm.assemble()
    a = [asm.block_csr_host(b, td.FAR)[2].copy() for b in range(asm.num_blocks())]
    asm.assemble()
    b = [asm.block_csr_host(b, td.FAR)[2] for b in range(asm.num_blocks())]
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_torus8192_graded_fullsize(td):
    """The batched uneven-block workload at full size (torus 8192 triangles,
    96 graded steps of ratio 1.02 on [0, 6], mixed precision), in the launch
    configuration bench.py times: the pattern fingerprint (entry count and
    sum of splitmix64(l M + j) mod 2^64) of every block over every row equals
    the oracle's; columns and values of 120 sampled blocks (seeded) on 3
    rows."""
    w = inputs.workload("torus8192g")
    rng = np.random.default_rng(0)
    from oracle.oracle import Oracle
    asm = td.Assembler(td.Mesh(w.verts, w.tris), td.TimeGrid(w.t), precision=1)
    asm.assemble()
    st = asm.stats()
    orc = Oracle(w.verts, w.tris, w.t, equidistant=False, psi_mode="interp")
    ob = orc.blocks()
    assert [(b[0], b[1]) for b in ob] == asm.blocks()
    nb, M = len(ob), w.M
    hs, nz = orc.pattern_hash(np.arange(nb))
    for b in range(nb):
        rp, col, _ = asm.block_csr_torch(b, td.FAR)
        h, n = device_fingerprint(rp, col, M)
        assert n == nz[b] and h == int(hs[b]), "pattern of block %d %s (all rows)" % (b, ob[b][:2])
    rows = np.array([5, 1111, 3333])
    blocks = np.sort(rng.choice(nb, size=120, replace=False))
    res = orc.assemble_rows(rows, blocks)
    errs = []
    for b in blocks:
        b = int(b)
        rp, col, val = asm.block_csr_torch(b, td.FAR)
        rpn, coln, valn = asm.block_csr_torch(b, td.NEAR)
        rp, rpn = rp.cpu().numpy(), rpn.cpu().numpy()
        num = den = 0.0
        for r, (c, f, n) in enumerate(res[b]):
            l = rows[r]
            gc = col[rp[l]:rp[l + 1]].cpu().numpy()
            assert np.array_equal(c, gc), "pattern block %d row %d" % (b, l)
            got = val[rp[l]:rp[l + 1]].double().cpu().numpy()
            nc = coln[rpn[l]:rpn[l + 1]].cpu().numpy()
            got[np.searchsorted(c, nc)] += valn[rpn[l]:rpn[l + 1]].cpu().numpy()
            num += np.sum((got - (f + n)) ** 2)
            den += np.sum((f + n) ** 2)
        errs.append((np.sqrt(num / den) if den > 0 else np.sqrt(num), b, ob[b][:2], np.sqrt(den)))
    rel, absmax = _worst(errs)
    print("torus8192g mixed: %d blocks, nnz %d, worst rel %.3e at %s, median %.3e, abs %.3e, %.1f ms "
          "(pattern %.1f, far %.1f, near %.1f, extract %.1f)"
          % (st["n_blocks"], st["nnz"], rel[0], rel[2], float(np.median([e[0] for e in errs])), absmax,
             st["ms_total"], st["ms_pattern"], st["ms_far"], st["ms_near"], st["ms_extract"]))
    assert rel[0] < TOL[1], rel
    assert absmax < TOL[1], absmax
