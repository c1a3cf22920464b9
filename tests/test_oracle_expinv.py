"""Pins of the oracle's second smooth step of the time basis, the one built
from h(s) = exp(-1/s): F(s) = h(s) / (h(s) + h(1 - s)), s = (x + 1)/2 on
|x| < 1 (the paper's Sec. 3 construction of the partition of unity with this
step in place of erf(2 artanh x)/2 + 1/2).

* Closed form: F at x = 1/2 is 1 / (1 + e^{-8/3}) (s = 3/4: h(3/4) = e^{-4/3},
  h(1/4) = e^{-4}); F(0) = 1/2; F'(0) = 1 (d/ds at s = 1/2 is 2).
* Symmetry F(1 - s) = 1 - F(s): f(-x) = 1 - f(x), f' even, f'' odd.
* f' and f'' against centred differences of f and f'.
* The partition of unity of Sec. 3 (mu_1..mu_N, equidistant and graded
  grids) holds with this step too, and psi = d^2 psi~/dr^2 (Eq. psis) for
  blocks of it.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, lib
from paper_1503_07221_gb300 import inputs


def _step(x):
    out = np.zeros(3)
    lib().or_step(1, float(x), out)
    return out


def test_step_closed_forms():
    assert abs(_step(0.5)[0] - 1.0 / (1.0 + math.exp(-8.0 / 3.0))) < 1e-15
    f0 = _step(0.0)
    assert abs(f0[0] - 0.5) < 1e-15 and abs(f0[1] - 1.0) < 1e-14 and abs(f0[2]) < 1e-14
    assert np.array_equal(_step(-1.0), [0.0, 0.0, 0.0]) and np.array_equal(_step(1.0), [1.0, 0.0, 0.0])


def test_step_symmetry_and_differences():
    xs = np.linspace(-0.97, 0.97, 41)
    h = 1e-5
    for x in xs:
        a, b = _step(x), _step(-x)
        assert abs(a[0] + b[0] - 1.0) < 1e-15
        assert abs(a[1] - b[1]) < 1e-12 * max(1.0, abs(a[1]))
        assert abs(a[2] + b[2]) < 1e-10 * max(1.0, abs(a[2]))
        fd1 = (_step(x + h)[0] - _step(x - h)[0]) / (2 * h)
        fd2 = (_step(x + h)[1] - _step(x - h)[1]) / (2 * h)
        assert abs(fd1 - a[1]) < 1e-7 * max(1.0, abs(a[1]))
        assert abs(fd2 - a[2]) < 1e-6 * max(1.0, abs(a[2]))


def _tiny(t, **kw):
    V, F = inputs.tiny_meshes()["tetra"]
    return Oracle(V, F, t, equidistant=False, psi_mode="direct", basis_kind=1, **kw)


@pytest.mark.parametrize("grid", ["eq", "graded"])
def test_partition_of_unity_expinv(grid):
    t = inputs.equidistant_grid(9, 2.0) if grid == "eq" else inputs.graded_grid(12, 1.1, 3.0)
    o = _tiny(t)
    o.set_first_kind(1)
    s = np.linspace(0.0, t[-1], 4001)
    tot = sum(o.mu(i, s)[:, 0] for i in range(t.size))
    assert np.abs(tot - 1.0).max() < 1e-15
    # the step differs from the paper's: the bump of mu_4 at the flank midpoint + 1/4
    x = 0.5
    s1 = 2 * 0.25 + (x + 1) / 2 * 0.25
    if grid == "eq":
        assert abs(o.mu(3, np.array([s1]))[0, 0] - 1.0 / (1.0 + math.exp(-8.0 / 3.0))) < 1e-15


def test_psi_second_derivative_expinv():
    o = _tiny(inputs.equidistant_grid(9, 2.0))
    r = np.linspace(0.31, 0.69, 9)
    h = 1e-4
    for kb, ib in ((4, 2), (4, 0), (8, 5)):
        p = o.psi(kb, ib, r)
        pt = o.psi(kb, ib, np.concatenate([r - h, r, r + h]))[:, 1].reshape(3, -1)
        fd = (pt[0] - 2 * pt[1] + pt[2]) / h ** 2
        scale = np.abs(p[:, 0]).max()
        assert scale > 0
        assert np.abs(fd - p[:, 0]).max() < 1e-5 * scale, (kb, ib)


def test_interpolant_follows_the_step():
    # the oracle's interpolant is sampled from the direct psi of the chosen step
    V, F = inputs.icosphere(1)
    t = inputs.equidistant_grid(9, 2.0)
    od = Oracle(V, F, t, psi_mode="direct", basis_kind=1)
    oi = Oracle(V, F, t, psi_mode="interp", basis_kind=1)
    o0 = Oracle(V, F, t, psi_mode="direct", basis_kind=0)
    r = np.linspace(0.01, 1.99, 41)
    for b in range(od.num_blocks()):
        d = od.psi_block(b, r)
        scale = np.abs(d).max()
        assert np.abs(oi.psi_block(b, r) - d).max() <= 1e-12 * scale
    assert np.abs(o0.psi_block(2, r) - od.psi_block(2, r)).max() > 1e-2 * np.abs(od.psi_block(2, r)).max()
