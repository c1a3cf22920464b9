"""tdbem_hessenberg_apply_noalloc (fixed device scratch, no allocation)
against tdbem_hessenberg_apply, both through the C ABI.

Collected last on purpose: it must pass in a fresh process and after every
other GPU test has run in the same process. Two calls in a row each match
the allocating entry point within 1e-12 of the largest |y| (the same kernel
runs on the same data in the same order, so they agree bit for bit in
practice), and the calls leave torch's allocation counters unchanged (the
library's allocator is torch's caching allocator here).
"""
import numpy as np
import pytest

from paper_1503_07221_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def _allocs():
    import torch
    s = torch.cuda.memory_stats()
    return s.get("allocation.all.allocated", 0), torch.cuda.memory_allocated()


@pytest.mark.parametrize("name,precision", [("sphere320", 0), ("sphere320", 1), ("sphere5120j", 1)])
def test_noalloc_matches_allocating_entry(td, name, precision):
    import torch
    if name == "sphere320":
        V, F = inputs.icosphere(2)
        t = inputs.equidistant_grid(17, 6.4)
    else:
        w = inputs.workload(name)
        V, F, t = w.verts, w.tris, w.t
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=precision)
    asm.assemble()
    x = torch.from_numpy(np.random.default_rng(7).standard_normal((t.size, V.shape[0]))).cuda()
    ref = asm.hessenberg_apply(x)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    scale = np.abs(ref).max()
    assert scale > 0
    ys = [torch.full_like(x, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    before = _allocs()
    for y in ys:
        asm.hessenberg_apply(x, y, noalloc=True)
    torch.cuda.synchronize()
    assert _allocs() == before, "the no-allocation entry point allocated device memory"
    for n, y in enumerate(ys):
        got = y.cpu().numpy()
        assert np.isfinite(got).all(), "call %d left entries unwritten" % n
        err = float(np.abs(got - ref).max())
        print("%s prec %d call %d: max |diff| / max |y| = %.3e" % (name, precision, n, err / scale))
        assert err <= 1e-12 * scale


def test_noalloc_rejects_oversize(td):
    import torch
    w = inputs.workload("sphere20480")
    t = inputs.equidistant_grid(257, 12.8)  # N*M = 257 * 10242 > 2^21
    asm = td.Assembler(td.Mesh(w.verts, w.tris), td.TimeGrid(t), precision=1)
    x = torch.zeros((t.size, w.M), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(td.TdbemError) as e:
        asm.hessenberg_apply(x, y, noalloc=True)
    assert e.value.code == td.E_INVALID_ARG
    assert "fixed scratch" in str(e.value)
