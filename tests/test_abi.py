"""The C-ABI library: it loads without a GPU, exports every symbol that
include/wh.h declares, and rejects bad arguments on the host before any
device work (no GPU needed for any check here)."""
import ctypes
import os
import re

import pytest

import paper_2110_13693_gb300 as wh
from paper_2110_13693_gb300 import build as whbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wh.h")


@pytest.fixture(scope="module")
def lib():
    whbuild.build()
    return wh.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|int32_t|uint32_t)\s+\**\s*(wh_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("wh_create_layout", "wh_eval_plans", "wh_destroy", "wh_get_last_status"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in wh.h but not exported"
        assert n in wh.SIGNATURES, f"{n} has no binding"


def test_create_layout_checks(lib):
    h = ctypes.c_void_p()

    def rc(*fields):
        return lib.wh_create_layout(ctypes.byref(wh.wh_layout_desc(*fields)), ctypes.byref(h))

    assert rc(10, 30, 3, 1, 3) == wh.WH_EINVAL          # odd cross-aisle width
    assert rc(0, 30, 3, 1, 2) == wh.WH_EINVAL
    assert rc(10, 0, 3, 1, 2) == wh.WH_EINVAL
    assert rc(10, 30, 0, 1, 2) == wh.WH_EINVAL
    assert rc(70000, 30, 3, 1, 2) == wh.WH_ERANGE       # too many aisles for the key
    assert rc(60000, 60000, 3, 1, 2) == wh.WH_ERANGE    # tour span bound
    assert lib.wh_create_layout(None, ctypes.byref(h)) == wh.WH_EINVAL
    assert rc(10, 30, 3, 1, 2) == wh.WH_OK and h.value
    lib.wh_destroy(h)
    lib.wh_destroy(None)


def test_eval_plans_host_checks(lib):
    h = ctypes.c_void_p()
    assert lib.wh_create_layout(ctypes.byref(wh.wh_layout_desc(10, 30, 3, 1, 2)), ctypes.byref(h)) == 0
    o = wh.wh_orders(0, 0, 1, 8, 0)
    p = wh.wh_plans(0, 0, 0, 0, 0, 0, 0, 0)
    c = wh.wh_costs(0, 0, 0, 0)
    call = lambda o, p, mask, c: lib.wh_eval_plans(h, ctypes.byref(o), ctypes.byref(p), mask, ctypes.byref(c), None)
    assert call(o, p, 0, c) == wh.WH_EINVAL              # empty routing mask
    assert call(o, p, 4, c) == wh.WH_EINVAL              # unknown routing bit
    assert call(wh.wh_orders(-1, 0, 1, 8, 0), p, 3, c) == wh.WH_EINVAL
    assert call(wh.wh_orders(0, 0, 1, 0, 0), p, 3, c) == wh.WH_EINVAL      # NULL order_off
    assert call(o, wh.wh_plans(1, 0, 0, 0, 0, 0, 0, 0), 3, c) == wh.WH_EINVAL  # NULL plan_tour_off
    assert call(wh.wh_orders(0, 0, 5, 8, 0), wh.wh_plans(0, 0, 0, 0, 3, 0, 0, 0), 3, c) == wh.WH_EINVAL  # 0 < stride < n_sku
    assert call(o, wh.wh_plans(0, 0, 1 << 33, 0, 0, 0, 0, 8), 3, c) == wh.WH_ERANGE
    assert call(o, p, 3, c) == wh.WH_OK                  # nothing to do: no device touched
    assert lib.wh_eval_plans(None, ctypes.byref(o), ctypes.byref(p), 3, ctypes.byref(c), None) == wh.WH_EINVAL
    lib.wh_destroy(h)


def test_status_without_device_use(lib):
    h = ctypes.c_void_p()
    assert lib.wh_create_layout(ctypes.byref(wh.wh_layout_desc(4, 4, 3, 1, 2)), ctypes.byref(h)) == 0
    v = ctypes.c_uint32(7)
    assert lib.wh_get_last_status(h, None, ctypes.byref(v)) == wh.WH_OK and v.value == 0
    assert lib.wh_get_last_status(h, None, None) == wh.WH_EINVAL
    lib.wh_destroy(h)
