"""The C-ABI library builds, loads on a machine without a GPU, and exports
every entry point include/pairgal.h declares (no compute calls)."""
import ctypes
import os
import re

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pairgal.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1705_03464_gb300 import build_lib
    path = build_lib.build(verbose=False)
    lib = ctypes.CDLL(path)
    names = _declared()
    assert "pg_forward" in names and "pg_plan_create" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_imports_and_status_strings():
    from paper_1705_03464_gb300 import build_lib
    build_lib.build(verbose=False)
    from paper_1705_03464_gb300 import pairgal
    assert pairgal.status_string(pairgal.PG_OK) == "ok"
    assert "memory" in pairgal.status_string(pairgal.PG_ERR_OOM)
    assert set(_declared()) <= set(n for n in dir(pairgal._lib) if n.startswith("pg_")) | set(_declared())


def test_binding_has_c_names():
    from paper_1705_03464_gb300 import build_lib
    build_lib.build(verbose=False)
    from paper_1705_03464_gb300 import pairgal
    for n in _declared():
        if n in ("pg_plan_create", "pg_plan_destroy", "pg_plan_reserve", "pg_workspace_bytes",
                 "pg_status_string", "pg_plan_set_profiling", "pg_plan_last_stats",
                 "pg_plan_create_shared"):
            continue   # wrapped by pairgal.Plan / status_string
        assert hasattr(pairgal, n), n


def test_binding_refuses_bad_buffers_before_the_call():
    """The binding checks dtype, device, contiguity and shape before a
    tensor's address reaches the library (the kernels read exactly the bytes
    the shape implies). All of these fail on the host, so no GPU is needed."""
    torch = pytest.importorskip("torch")
    from paper_1705_03464_gb300 import build_lib
    build_lib.build(verbose=False)
    from paper_1705_03464_gb300 import pairgal as pg
    edges = (0.0, 1.0, 2.0)
    cases = [
        (torch.zeros((10, 3), dtype=torch.float64), None),          # host tensor
        (torch.zeros((10, 3), dtype=torch.float32), None),          # wrong dtype
        (torch.zeros((3, 10), dtype=torch.float64).t(), None),      # strided view
        (torch.zeros((10, 2), dtype=torch.float64), None),          # wrong shape
        (torch.zeros((10, 3)).numpy(), None),                       # not a tensor
    ]
    for pos, w in cases:
        with pytest.raises(pg.PairgalError) as e:
            pg.pg_pair_counts_static(pos, w, 10.0, edges, 1)
        assert e.value.status == pg.PG_ERR_INVALID_ARG
    with pytest.raises(pg.PairgalError) as e:
        pg._dev(torch.zeros(5, dtype=torch.float64), "w", "f32", (5,))
    assert e.value.status == pg.PG_ERR_INVALID_ARG
    # host arrays: a short weight array is refused, a float64 one converted
    with pytest.raises(pg.PairgalError):
        pg._host_arr(np.zeros(4), "w", np.float32, (5,))
    a = pg._host_arr(np.zeros(5), "w", np.float32, (5,))
    assert a.dtype == np.float32 and a.flags.c_contiguous
