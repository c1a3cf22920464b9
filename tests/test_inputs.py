"""Seeded synthetic inputs shared by the CUDA path and the oracle: meshes are
closed, consistently and outward oriented surfaces of the stated sizes; the
jitter and time grids follow their stated recipes; splitmix64 reproduces
its published sequence."""
import numpy as np
import pytest

from paper_1503_07221_gb300 import inputs


def _edges_consistent(F):
    """Every undirected edge is used by exactly two triangles, once in each
    direction (closed, consistently oriented 2-manifold)."""
    d = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    fwd = {tuple(e) for e in d}
    assert len(fwd) == d.shape[0], "a directed edge occurs twice"
    for a, b in fwd:
        assert (b, a) in fwd, "edge (%d, %d) has no twin" % (a, b)
    return d.shape[0] // 2


def test_splitmix64_published_sequence():
    # splitmix64 started at state 0: 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4,
    # 0x06c45d188009454f (Steele, Lea, Flood 2014); the doubles keep the top 53 bits
    u = inputs.splitmix64_uniform(0, 3)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(x * 2.0 ** 53) for x in u] == [w >> 11 for w in want]


@pytest.mark.parametrize("level", [0, 1, 2, 3])
def test_icosphere(level):
    V, F = inputs.icosphere(level)
    assert F.shape == (20 * 4 ** level, 3) and V.shape == (10 * 4 ** level + 2, 3)
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-15)
    ne = _edges_consistent(F)
    assert V.shape[0] - ne + F.shape[0] == 2  # Euler characteristic of the sphere
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, c - a)
    assert (np.einsum("ij,ij->i", n, a + b + c) > 0).all()  # outward


def test_torus():
    nM, nm = 16, 8
    V, F = inputs.torus(1.0, 0.4, nM, nm)
    assert F.shape == (2 * nM * nm, 3) and V.shape == (nM * nm, 3)
    rho = np.hypot(V[:, 0], V[:, 1])
    assert np.allclose((rho - 1.0) ** 2 + V[:, 2] ** 2, 0.16, atol=1e-14)
    ne = _edges_consistent(F)
    assert V.shape[0] - ne + F.shape[0] == 0  # Euler characteristic of the torus
    # enclosed volume by the divergence theorem: positive for outward normals,
    # below the smooth torus's 2 pi^2 R r^2 (an inscribed polyhedron; 88 % at 16 x 8)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    assert 0.8 * 2 * np.pi ** 2 * 0.16 < vol < 2 * np.pi ** 2 * 0.16


def test_jitter_recipe():
    V, F = inputs.icosphere(2)
    h = inputs.mean_edge_length(V, F)
    J = inputs.jitter(V, F, 0.01, 0)
    d = J - V
    assert np.abs(d).max() <= 0.01 * h and np.abs(d).max() > 0.009 * h
    assert np.array_equal(J, inputs.jitter(V, F, 0.01, 0))
    assert not np.array_equal(J, inputs.jitter(V, F, 0.01, 1))
    u = inputs.splitmix64_uniform(0, V.size).reshape(V.shape)
    assert np.allclose(d, (2 * u - 1) * 0.01 * h, rtol=0, atol=4e-16)


def test_time_grids():
    t = inputs.equidistant_grid(17, 4.0)
    assert t.size == 17 and t[0] == 0.0 and t[-1] == 4.0 and np.allclose(np.diff(t), 0.25)
    g = inputs.graded_grid(96, 1.02, 6.0)
    d = np.diff(g)
    assert g.size == 97 and g[0] == 0.0 and abs(g[-1] - 6.0) < 1e-13
    assert np.allclose(d[1:] / d[:-1], 1.02, rtol=1e-12)
    assert (d > 0).all()


@pytest.mark.parametrize("name,E,M,N", [("sphere320", 320, 162, 17), ("sphere5120j", 5120, 2562, 65),
                                        ("torus2048g", 2048, 1024, 97), ("sphere20480", 20480, 10242, 129)])
def test_named_workloads(name, E, M, N):
    w = inputs.workload(name)
    assert (w.E, w.M, w.N) == (E, M, N)
    assert w.tris.dtype == np.int32 and w.verts.dtype == np.float64
    assert w.tris.min() == 0 and w.tris.max() == M - 1
