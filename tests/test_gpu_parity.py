"""GPU parity: the CUDA assembler through the C ABI against the FP64 oracle.

Per unique block: the sparsity pattern must be identical (row offsets and
sorted columns), and the values must agree in relative Frobenius norm,
||A_gpu - A_oracle||_F / ||A_oracle||_F with A = far + near, and the far part
(element pairs without a shared vertex) and the near part (Sauter-Schwab
pairs) separately against the same denominator.
Tolerances: FP64 path 1e-10 (table and quadrature rounding only), mixed
path 1e-6 (FP32 far field).
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


def _dense(M, rp, col, val):
    A = np.zeros((M, M))
    for l in range(M):
        A[l, col[rp[l]:rp[l + 1]]] = val[rp[l]:rp[l + 1]]
    return A


def _compare(td, V, F, t, precision, rows=None):
    from oracle.oracle import Oracle
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=precision)
    asm.assemble()
    orc = Oracle(V, F, t, psi_mode="interp")
    ob = orc.blocks()
    assert [(b[0], b[1]) for b in ob] == asm.blocks()
    M = V.shape[0]
    rows = np.arange(M) if rows is None else np.asarray(rows)
    res = orc.assemble_rows(rows, np.arange(len(ob)))
    errs = []
    for b in range(len(ob)):
        rp, col, vf = asm.block_csr_host(b, td.FAR)
        rpn, coln, vn = asm.block_csr_host(b, td.NEAR)
        Af = _dense(M, rp, col, vf.astype(np.float64))[rows]
        An = _dense(M, rpn, coln, vn)[rows]
        Rf = np.zeros((rows.size, M)); Rn = np.zeros((rows.size, M))
        for r, (c, f, n) in enumerate(res[b]):
            l = rows[r]
            assert np.array_equal(c, col[rp[l]:rp[l + 1]]), "pattern of block %d row %d" % (b, l)
            Rf[r, c] = f; Rn[r, c] = n
        # each part is measured against the norm of the whole block: near the
        # end of a support the far part alone can be ~1e-24 of the block
        nr = np.linalg.norm(Rf + Rn)
        for A, R, name in ((Af, Rf, "far"), (An, Rn, "near"), (Af + An, Rf + Rn, "sum")):
            e = np.linalg.norm(A - R) / nr if nr > 0 else np.linalg.norm(A)
            errs.append((e, b, name, ob[b][:2]))
    return asm, errs


@pytest.mark.parametrize("precision", [0, 1])
def test_sphere80_n9(td, precision):
    V, F = inputs.icosphere(1)
    _, errs = _compare(td, V, F, inputs.equidistant_grid(9, 2.0), precision)
    worst = max(errs)
    assert worst[0] < TOL[precision], worst


@pytest.mark.parametrize("precision", [0, 1])
def test_sphere320_n17(td, precision):
    # the plain-method workload: 320 triangles, 16 steps of 0.25 on [0, 4]
    V, F = inputs.icosphere(2)
    _, errs = _compare(td, V, F, inputs.equidistant_grid(17, 4.0), precision)
    worst = max(errs)
    assert worst[0] < TOL[precision], worst


@pytest.mark.parametrize("precision", [0, 1])
def test_jittered_sphere_small_n(td, precision):
    # N = 5: the last-row/first-column special block (N-1, 0) is live
    V, F = inputs.icosphere(1)
    V = inputs.jitter(V, F, 0.05, 7)
    _, errs = _compare(td, V, F, inputs.equidistant_grid(5, 2.0), precision)
    worst = max(errs)
    assert worst[0] < TOL[precision], worst


def test_deterministic(td):
    V, F = inputs.icosphere(2)
    t = inputs.equidistant_grid(17, 4.0)
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=1)
    asm.assemble()
    a = [asm.block_csr_host(b, td.FAR)[2].copy() for b in range(asm.num_blocks())]
    asm.assemble()
    b = [asm.block_csr_host(b, td.FAR)[2] for b in range(asm.num_blocks())]
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_too_coarse_mesh_is_rejected(td):
    V, F = inputs.icosphere(0)
    with pytest.raises(td.TdbemError) as e:
        td.Assembler(td.Mesh(V, F), td.TimeGrid(inputs.equidistant_grid(33, 2.0)))
    assert e.value.code == 8


def test_graph_replay_is_identical(td):
    """The second assembly replays the recorded CUDA graph: same values, bit
    for bit, and the same borrowed pointers."""
    V, F = inputs.icosphere(2)
    t = inputs.equidistant_grid(17, 6.4)
    for prec in (0, 1):
        asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=prec)
        asm.assemble()
        first = [asm.block_csr_host(b, w) for b in range(asm.num_blocks()) for w in (td.FAR, td.NEAR)]
        ptrs = [asm.block_csr_device(b, td.FAR) for b in range(asm.num_blocks())]
        s1 = asm.stats()
        for _ in range(2):
            asm.assemble()
        s2 = asm.stats()
        assert s2["graph_replays"] == 2 and s1["graph_replays"] == 0
        again = [asm.block_csr_host(b, w) for b in range(asm.num_blocks()) for w in (td.FAR, td.NEAR)]
        for (r1, c1, v1), (r2, c2, v2) in zip(first, again):
            assert np.array_equal(r1, r2) and np.array_equal(c1, c2) and np.array_equal(v1, v2)
        assert ptrs == [asm.block_csr_device(b, td.FAR) for b in range(asm.num_blocks())]
        assert s2["nnz"] == s1["nnz"] and s2["ms_far"] > 0


def test_measured_fma_peaks(td):
    """The roofline denominators: packed FP32 and FP64 FMA throughput."""
    p32, p64 = td.measure_fma_peaks()
    print("FMA peaks: fp32 %.1f TFLOP/s, fp64 %.2f TFLOP/s" % (p32, p64))
    assert 10.0 < p32 < 200.0 and 0.05 < p64 < 100.0
