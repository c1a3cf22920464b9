"""GPU retarded double layer potential (tdbem_double_layer, Eq.
RetardedPotential) through the C ABI.

* Parity with the FP64 oracle (Oracle.double_layer: the same collapsed Gauss
  product rule per triangle) for a seeded density on the 320-triangle
  sphere, points inside and outside, times across the whole grid: both sides
  are FP64, so they agree to rounding (1e-11 of the largest |u|).
* Gauss's law, fixed by the mathematics rather than the oracle: once every
  retarded time t - |x - y| lies beyond the last grid point, only the last
  time basis function (equal to 1 there) carries the density, d_t phi = 0,
  and u(x) = -1/(4 pi) int n_y.(x - y)/|x - y|^3 is the solid angle: 1
  inside the closed surface, 0 outside (1e-10 with 8 x 8 points per
  triangle at these distances).
* Causality: before the first retarded time reaches the surface, u = 0.
"""
import numpy as np
import pytest

from paper_1503_07221_gb300 import inputs

pytestmark = pytest.mark.gpu

T9 = inputs.equidistant_grid(9, 2.0)
X = np.array([[0, 0, 1.5], [0.3, -1.2, 0.9], [0, 0, 0.2], [0.1, 0.3, -0.4], [1.1, 0.7, -0.6]])
INSIDE = np.array([0, 0, 1, 1, 0])


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


def _run(td, V, F, t, alpha, X, times, n):
    import torch
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(t))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    u = asm.double_layer(dev(alpha), dev(X), dev(times), n=n)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def test_potential_matches_oracle(td):
    from oracle.oracle import Oracle
    V, F = inputs.icosphere(2)
    alpha = np.random.default_rng(11).standard_normal((T9.size, V.shape[0]))
    times = np.array([0.7, 1.3, 1.95, 2.6, 3.4])
    got = _run(td, V, F, T9, alpha, X, times, 4)
    ref = Oracle(V, F, T9, psi_mode="direct").double_layer(alpha, X, times, n=4)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print("potential vs oracle: max |diff| / max |u| = %.3e" % err)
    assert err < 1e-11


def test_potential_gauss_law_and_causality(td):
    V, F = inputs.icosphere(2)
    alpha = np.random.default_rng(5).standard_normal((T9.size, V.shape[0]))
    alpha[-1] = 1.0  # the last time function carries density 1
    u = _run(td, V, F, T9, alpha, X, np.array([5.0]), 8)[:, 0]  # 5 - |x - y| > T = 2 for every y
    assert np.abs(u - INSIDE).max() < 1e-10, u
    u0 = _run(td, V, F, T9, alpha, X[:2], np.array([0.45]), 8)  # exterior points 0.5 from the sphere
    assert np.array_equal(u0, np.zeros_like(u0))


def test_potential_rejects_bad_arguments(td):
    import torch
    V, F = inputs.icosphere(1)
    asm = td.Assembler(td.Mesh(V, F), td.TimeGrid(T9))
    a = torch.zeros((T9.size, V.shape[0]), dtype=torch.float64, device="cuda")
    x = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    tt = torch.ones(1, dtype=torch.float64, device="cuda")
    with pytest.raises(td.TdbemError) as e:
        asm.double_layer(a, x, tt, n=0)
    assert e.value.code == td.E_INVALID_ARG
