"""The C-ABI library builds, loads without a GPU and exports what the header declares."""
import ctypes
import os
import re

import pytest

from paper_2009_05264_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_binding_exports():
    assert declared_functions() == set(lbm.EXPORTS)


def test_library_loads_and_exports_every_symbol():
    L = lbm.load()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_struct_layout_matches_header():
    L = lbm.load()
    p = lbm.LbmParams()
    L.lbm_default_params(ctypes.byref(p))
    assert p.size == ctypes.sizeof(lbm.LbmParams)
    assert p.beta == 1.16 and p.c0 == 6.0 and p.a == 2.0 / 49.0 and p.b == 2.0 / 21.0
    assert p.G_wet == pytest.approx(9.0 * (1.0 + p.beta) * p.G)


def test_required_bytes_and_host_only_calls():
    L = lbm.load()
    n1 = L.lbm_required_bytes(1000, 100, lbm.FP32)
    n2 = L.lbm_required_bytes(1000, 100, lbm.FP64)
    assert n1 >= 4 * 9 * 1000 * 100 * 4 and n2 >= 4 * 9 * 1000 * 100 * 8
    assert L.lbm_required_bytes(0, 10, lbm.FP32) == 0
    assert L.lbm_status_string(3) == b"lattice unstable"
    assert L.lbm_destroy(None) == 0
    p = lbm.LbmParams()
    L.lbm_default_params(ctypes.byref(p))
    assert L.lbm_critical_temperature(ctypes.byref(p)) == pytest.approx(0.0778 * p.a / (0.45724 * p.b * p.R))


def test_create_rejects_bad_sizes_without_touching_a_gpu():
    L = lbm.load()
    h = ctypes.c_void_p()
    assert L.lbm_create(ctypes.byref(h), 0, 10, lbm.FP32, 0, None) == 1
    assert L.lbm_create(ctypes.byref(h), 10, 10, 7, 0, None) == 1
    assert L.lbm_create_ex(ctypes.byref(h), 10, 10, lbm.FP32, 0, None, None, 0) == 1
