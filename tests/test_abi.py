"""The C-ABI library builds, loads and exports every symbol declared in
include/tdbem.h; host-side argument validation returns the documented codes
(no GPU needed: these calls do not touch the device)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1503_07221_gb300 import build, tdbem
    build.build()
    return tdbem.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "tdbem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tdbem_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    from paper_1503_07221_gb300 import tdbem
    assert sorted(tdbem.exported_symbols()) == sorted(set(tdbem.exported_symbols()) & set(names))


def test_mesh_validation(L):
    from paper_1503_07221_gb300 import tdbem
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    with pytest.raises(tdbem.TdbemError) as e:
        tdbem.Mesh(V, np.array([[0, 1, 7]], np.int32))
    assert e.value.code == 2
    with pytest.raises(tdbem.TdbemError) as e:
        tdbem.Mesh(V, np.array([[0, 1, 1]], np.int32))
    assert e.value.code == 2
    Vn = V.copy(); Vn[2, 1] = np.nan
    with pytest.raises(tdbem.TdbemError) as e:
        tdbem.Mesh(Vn, np.array([[0, 1, 2]], np.int32))
    assert e.value.code == 2
    Vd = V.copy(); Vd[2] = [2, 0, 0]  # collinear: zero area
    with pytest.raises(tdbem.TdbemError) as e:
        tdbem.Mesh(Vd, np.array([[0, 1, 2]], np.int32))
    assert e.value.code == 2
    m = tdbem.Mesh(V, np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32))
    assert m.E == 4


def test_timegrid_validation(L):
    from paper_1503_07221_gb300 import tdbem
    for bad in ([0.0, 1.0], [0.1, 0.5, 1.0], [0.0, 0.5, 0.5, 1.0], [0.0, 0.7, 0.6]):
        with pytest.raises(tdbem.TdbemError) as e:
            tdbem.TimeGrid(np.array(bad))
        assert e.value.code == 3
    # temporal degree p = 0, 1, 2 (Eq. BasisFunctions); 3 is not built
    for p in (0, 1, 2):
        tdbem.TimeGrid(np.linspace(0, 1, 5), p=p)
    with pytest.raises(tdbem.TdbemError) as e:
        tdbem.TimeGrid(np.linspace(0, 1, 5), p=3)
    assert e.value.code == 8
    with pytest.raises(tdbem.TdbemError) as e:
        tdbem.TimeGrid(np.linspace(0, 1, 5), c=-1.0)
    assert e.value.code == 1
    tdbem.TimeGrid(np.linspace(0, 1, 5))


def test_null_arguments(L):
    out = C.c_void_p()
    assert L.tdbem_mesh_create(None, 3, None, 1, C.byref(out)) == 1
    assert L.tdbem_timegrid_create(None, 5, 0, 0, 1.0, C.byref(out)) == 1
    n = C.c_int64()
    assert L.tdbem_num_blocks(None, C.byref(n)) == 1
    assert L.tdbem_last_error()
