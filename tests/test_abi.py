"""CPU checks of the native boundary: the library builds, loads, and exports
every function include/amm.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(amm_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_0901_4107_gb300 import _build
    path = _build.build()
    L = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    from paper_0901_4107_gb300 import amm
    names = _declared()
    missing = [n for n in sorted(names) if not hasattr(amm, n) and n not in amm._SIGS]
    assert not missing, missing


def test_create_rejects_bad_input_before_touching_the_device():
    """Host-side validation runs before any CUDA call, so it works on CPU."""
    import numpy as np
    from paper_0901_4107_gb300 import amm
    from harness import ics
    P = ics.turbulent_3d(6, seed=1)
    T = P.tess
    Q = P.conserved()
    bad_cells = T.cells.copy()
    bad_cells[3, 1] = T.n_cells + 5
    with pytest.raises(amm.AmmError) as e:
        amm.amm_create(3, T.points, bad_cells, T.shift, T.area, T.centroid, T.box, Q, P.gamma)
    assert e.value.code == amm.AMM_ERR_INVALID_ARG
    Qn = Q.copy()
    Qn[7, 0] = -1.0
    with pytest.raises(amm.AmmError) as e:
        amm.amm_create(3, T.points, T.cells, T.shift, T.area, T.centroid, T.box, Qn, P.gamma)
    assert e.value.code == amm.AMM_ERR_NONPOSITIVE_STATE
    Qnan = Q.copy()
    Qnan[2, 4] = np.nan
    with pytest.raises(amm.AmmError) as e:
        amm.amm_create(3, T.points, T.cells, T.shift, T.area, T.centroid, T.box, Qnan, P.gamma)
    assert e.value.code == amm.AMM_ERR_INVALID_ARG
    area = T.area.copy()
    area[0] = -1.0
    with pytest.raises(amm.AmmError) as e:
        amm.amm_create(3, T.points, T.cells, T.shift, area, T.centroid, T.box, Q, P.gamma)
    assert e.value.code == amm.AMM_ERR_INVALID_ARG
