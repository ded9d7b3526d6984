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


def test_next_row_entry_points_host_checks(lib):
    """Explicit routes, K-means slotting, occupancy bits, 16-bit widening and
    batch formation reject bad arguments (and do nothing for empty work)
    before any device call."""
    h = ctypes.c_void_p()
    assert lib.wh_create_layout(ctypes.byref(wh.wh_layout_desc(10, 30, 3, 1, 2)), ctypes.byref(h)) == 0
    big = ctypes.c_void_p()
    assert lib.wh_create_layout(ctypes.byref(wh.wh_layout_desc(300, 30, 3, 1, 2)), ctypes.byref(big)) == 0
    o = wh.wh_orders(2, 4, 600, 16, 32)          # pointer values only: nothing is dereferenced
    p = wh.wh_plans(1, 2, 4, 48, 0, 64, 80, 96)
    P = ctypes.c_void_p
    # routes
    r = lambda hh, n, tours, pts, npt, ln: lib.wh_routes(hh, ctypes.byref(o), ctypes.byref(p), P(tours), n, 256,
                                                        P(pts), P(npt), P(ln), None)
    assert r(None, 1, 16, 16, 16, 16) == wh.WH_EINVAL
    assert r(h, -1, 16, 16, 16, 16) == wh.WH_EINVAL
    assert r(h, 0, 0, 0, 0, 0) == wh.WH_OK
    assert r(h, 3, 0, 16, 16, 16) == wh.WH_EINVAL   # NULL tour list
    assert r(h, 3, 16, 16, 0, 16) == wh.WH_EINVAL   # NULL counts
    # K-means slotting
    def km(hh, signs, fw, k, init, u, iters, x_out=0):
        return lib.wh_kmeans_slotting(hh, ctypes.byref(o), P(signs), fw, k, P(init), P(u), iters, P(x_out), None,
                                      P(16), P(16), P(16), None)
    assert km(None, 16, 64, 8, 16, 0, 5) == wh.WH_EINVAL
    assert km(h, 0, 64, 8, 16, 0, 5) == wh.WH_EINVAL          # NULL signs
    assert km(h, 16, 64, 8, 0, 0, 5) == wh.WH_EINVAL          # neither seeds nor draws
    assert km(h, 16, 64, 0, 16, 0, 5) == wh.WH_EINVAL         # k = 0
    assert km(h, 16, 64, 8, 16, 0, -1) == wh.WH_EINVAL        # negative rounds
    assert km(h, 16, -1, 8, 16, 0, 5) == wh.WH_EINVAL
    assert km(h, 8, 64, 8, 16, 0, 5) == wh.WH_EINVAL          # signs not 16-byte aligned
    assert km(h, 16, 64, 8, 16, 0, 5, x_out=24) == wh.WH_EINVAL
    assert km(h, 16, 64, 257, 16, 0, 5) == wh.WH_ERANGE       # more than 256 clusters
    assert km(h, 16, 257, 8, 16, 0, 5) == wh.WH_ERANGE        # frequency weight above 256
    small = ctypes.c_void_p()
    assert lib.wh_create_layout(ctypes.byref(wh.wh_layout_desc(2, 10, 3, 1, 2)), ctypes.byref(small)) == 0
    assert km(small, 16, 64, 8, 16, 0, 5) == wh.WH_ERANGE     # 600 SKUs, 40 locations
    lib.wh_destroy(small)
    # occupancy bits
    occ = lambda plans: lib.wh_occupancy(h, ctypes.byref(o), ctypes.byref(plans), None)
    assert occ(wh.wh_plans(1, 2, 4, 48, 0, 64, 80, 96, 112)) == wh.WH_EINVAL      # shared slotting
    assert occ(wh.wh_plans(1, 2, 4, 48, 600, 64, 80, 96, 0)) == wh.WH_EINVAL      # no bit array
    assert occ(wh.wh_plans(0, 0, 0, 48, 600, 64, 80, 96, 0)) == wh.WH_OK          # no plans
    assert lib.wh_occupancy(None, ctypes.byref(o), ctypes.byref(p), None) == wh.WH_EINVAL
    # screen diagnostics: nothing screened on a fresh layout
    n_t, pt, pc, pf = ctypes.c_int64(7), ctypes.c_void_p(1), ctypes.c_void_p(1), ctypes.c_void_p(1)
    assert lib.wh_surrogate_screen_trace(h, ctypes.byref(n_t), ctypes.byref(pt), ctypes.byref(pc),
                                         ctypes.byref(pf)) == wh.WH_OK
    assert n_t.value == 0 and not pt.value and not pc.value and not pf.value
    assert lib.wh_surrogate_screen_trace(None, ctypes.byref(n_t), ctypes.byref(pt), ctypes.byref(pc),
                                         ctypes.byref(pf)) == wh.WH_EINVAL
    # widening
    assert lib.wh_widen_u16(P(16), P(16), -1, None) == wh.WH_EINVAL
    assert lib.wh_widen_u16(None, P(16), 8, None) == wh.WH_EINVAL
    assert lib.wh_widen_u16(None, None, 0, None) == wh.WH_OK
    # batch formation: 16-bit keys need at most 255 aisles
    bg = lambda hh, n_maps, mo: lib.wh_batch_grow(hh, ctypes.byref(o), P(48), 0, n_maps, mo, 0, P(16), P(16),
                                                  P(16), None)
    assert bg(big, 1, 8) == wh.WH_ERANGE
    assert bg(h, -1, 8) == wh.WH_EINVAL
    assert bg(h, 1, -1) == wh.WH_EINVAL
    assert bg(h, 0, 8) == wh.WH_OK
    lib.wh_destroy(big)
    lib.wh_destroy(h)
