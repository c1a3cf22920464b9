"""The device Chebyshev tables of psi and psi~ (Sec. 3.1) against the
oracle's direct 1-D Gauss-Legendre quadrature of Eq. psis, 1000 points per
panel of every unique block, through tdbem_psi_table. Error relative to the
block's max |psi| (and max |psi~| for psi~):
  FP64 set (4 sub-panels of degree 32 per time step): <= 1e-12;
  FP32 set (one panel of degree 32 per time step, FP32 coefficients with the
  residuals of the four leading ones): <= 2e-8 (measured 1.1e-8: the FP32
  rounding of the coefficients n >= 4 and the degree-32 truncation on a
  whole step).
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


@pytest.mark.parametrize("level,N,T", [(1, 9, 2.0), (2, 17, 4.0)])
def test_tables_against_direct_psi(td, level, N, T):
    import torch
    from oracle.oracle import Oracle
    V, F = inputs.icosphere(level)
    t = inputs.equidistant_grid(N, T)
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t), precision=td.PREC_MIXED)
    asm.assemble()
    orc = Oracle(V, F, t, psi_mode="direct")
    dt = t[1] - t[0]
    worst = {0: 0.0, 1: 0.0}
    for b, (kb, ib, m2, m1, a, bb) in enumerate(orc.blocks()):
        npan = int(round((bb - a) / dt))
        # 1000 points per time-step panel, strictly inside each panel
        u = (np.arange(1000) + 0.5) / 1000
        r = np.concatenate([a + (p + u) * dt for p in range(npan)])
        ref = orc.psi(kb, ib, r)
        scale = np.abs(ref).max(axis=0)
        assert scale.min() > 0
        rd = torch.from_numpy(r).cuda()
        for which in (0, 1):
            got = asm.psi_table(b, rd, which).cpu().numpy()
            err = float((np.abs(got - ref).max(axis=0) / scale).max())
            worst[which] = max(worst[which], err)
    print("level %d N %d: tables vs direct psi, FP64 set %.3e, FP32 set %.3e" % (level, N, worst[0], worst[1]))
    assert worst[0] <= 1e-12 and worst[1] <= 2e-8
