"""Seeded synthetic workloads for the warehouse plan evaluator.

Inputs only: this package builds order books, slottings, candidate plans and
moves with the C generator in ``gen.c`` and returns numpy arrays.  It holds no
tour-cost arithmetic; the CPU oracle and the CUDA path both consume what it
writes.  The five workload presets follow the paper's problem statement
(Sec. 5: layout, product position x, order history o, picking lists) at the
scale stated in Sec. 1 (~4,000 orders, ~10,000 items a day, up to 200,000
locations).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libwh_gen.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile gen.c into libwh_gen.so beside it (plain gcc, no -march)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.gen_orders.restype = ctypes.c_int64
            lib.gen_orders.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_double, i32p, i32p, ctypes.c_int64]
            lib.gen_orders_cat.restype = ctypes.c_int64
            lib.gen_orders_cat.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_double,
                                           i32p, i32p, ctypes.c_int64]
            lib.gen_signs.restype = ctypes.c_int
            lib.gen_signs.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
            lib.gen_slot_random.restype = ctypes.c_int
            lib.gen_slot_random.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, i32p]
            lib.gen_slot_abc.restype = ctypes.c_int
            lib.gen_slot_abc.argtypes = [ctypes.c_uint64] + [ctypes.c_int32] * 6 + [ctypes.c_double, i32p]
            lib.gen_plans.restype = ctypes.c_int64
            lib.gen_plans.argtypes = [ctypes.c_uint64, ctypes.c_int32, i32p, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p,
                                      ctypes.c_int64]
            lib.gen_moves.restype = ctypes.c_int
            lib.gen_moves.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_int32, i32p]
            lib.gen_relocations.restype = ctypes.c_int
            lib.gen_relocations.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, i32p,
                                            ctypes.c_int32, ctypes.c_int32, i32p]
            lib.gen_instance_param.restype = ctypes.c_int32
            lib.gen_instance_param.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_int32]
            lib.gen_stream_word.restype = ctypes.c_uint64
            lib.gen_stream_word.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _check(rc, what):
    if rc < 0:
        raise ValueError(f"{what} failed with code {rc}")
    return rc


# --------------------------------------------------------------------------- data

@dataclass
class Layout:
    """Single-block warehouse geometry (integer units).

    n_aisles parallel aisles at pitch ``aisle_pitch``; ``slots_per_side``
    slots on each side of an aisle at pitch ``slot_pitch``; front and back
    cross-aisles of width ``cross_aisle_width``; depot at the front of aisle 0.
    Location id ``loc = (aisle*2 + side)*slots_per_side + k``.
    """
    n_aisles: int
    slots_per_side: int
    aisle_pitch: int = 3
    slot_pitch: int = 1
    cross_aisle_width: int = 2

    @property
    def n_loc(self) -> int:
        return self.n_aisles * 2 * self.slots_per_side

    def loc(self, aisle: int, k: int, side: int = 0) -> int:
        return (aisle * 2 + side) * self.slots_per_side + k


@dataclass
class Instance:
    """One warehouse instance with its order book, slotting and plans (CSR)."""
    layout: Layout
    n_sku: int
    order_off: np.ndarray      # int32 [n_orders+1]
    line_sku: np.ndarray       # int32 [n_lines]
    slot_map: np.ndarray       # int32 [n_sku] (shared by all plans)
    plan_tour_off: np.ndarray  # int32 [n_plans+1]
    tour_off: np.ndarray       # int32 [n_tours+1], indexes order_seq
    order_seq: np.ndarray      # int32 [n_plans*n_orders]
    meta: dict = field(default_factory=dict)

    @property
    def n_orders(self) -> int:
        return int(self.order_off.shape[0] - 1)

    @property
    def n_lines(self) -> int:
        return int(self.line_sku.shape[0])

    @property
    def n_plans(self) -> int:
        return int(self.plan_tour_off.shape[0] - 1)

    @property
    def n_tours(self) -> int:
        return int(self.tour_off.shape[0] - 1)

    def tour_lines(self) -> np.ndarray:
        """Line count of every tour (orders' line counts summed)."""
        sizes = np.diff(self.order_off).astype(np.int64)
        cs = np.concatenate([[0], np.cumsum(sizes[self.order_seq])])
        return (cs[self.tour_off[1:]] - cs[self.tour_off[:-1]]).astype(np.int64)

    def subset_plans(self, plans) -> "Instance":
        """A copy holding only the listed plans (re-based CSR)."""
        plans = np.asarray(plans, dtype=np.int64)
        pto, to, segs, base = [0], [0], [], 0
        for p in plans:
            t0, t1 = int(self.plan_tour_off[p]), int(self.plan_tour_off[p + 1])
            s0, s1 = int(self.tour_off[t0]), int(self.tour_off[t1])
            segs.append(self.order_seq[s0:s1])
            to.extend((self.tour_off[t0 + 1:t1 + 1].astype(np.int64) - s0 + base).tolist())
            base += s1 - s0
            pto.append(pto[-1] + (t1 - t0))
        seq = np.concatenate(segs) if segs else np.zeros(0, np.int32)
        return Instance(self.layout, self.n_sku, self.order_off, self.line_sku, self.slot_map,
                        np.asarray(pto, np.int32), np.asarray(to, np.int32),
                        np.ascontiguousarray(seq, dtype=np.int32), dict(self.meta))


# ---------------------------------------------------------------------- generators

def gen_orders(seed: int, n_orders: int, n_sku: int, max_lines: int, p_geom: float,
               zipf_s: float = 0.0):
    lib = _load()
    off = np.zeros(n_orders + 1, np.int32)
    cap = max(1, n_orders * max_lines)
    lines = np.zeros(cap, np.int32)
    n = _check(lib.gen_orders(seed, n_orders, n_sku, max_lines, p_geom, zipf_s, _p(off), _p(lines), cap),
               "gen_orders")
    return off, np.ascontiguousarray(lines[:n])


def gen_orders_cat(seed: int, n_orders: int, n_sku: int, max_lines: int, p_geom: float, zipf_s: float,
                   n_cat: int, p_in: float):
    """Orders with categories (see gen.c): SKU s in category s mod n_cat; an
    order's lines come from its category with probability p_in."""
    lib = _load()
    off = np.zeros(n_orders + 1, np.int32)
    cap = max(1, n_orders * max_lines)
    lines = np.zeros(cap, np.int32)
    n = _check(lib.gen_orders_cat(seed, n_orders, n_sku, max_lines, p_geom, zipf_s, n_cat, p_in, _p(off),
                                  _p(lines), cap), "gen_orders_cat")
    return off, np.ascontiguousarray(lines[:n])


def gen_signs(seed: int, shape) -> np.ndarray:
    """int8 array of the given shape with entries in {-1, +1}."""
    out = np.zeros(int(np.prod(shape)), np.int8)
    _check(_load().gen_signs(seed, out.shape[0], out.ctypes.data), "gen_signs")
    return out.reshape(shape)


def gen_slot_random(seed: int, n_sku: int, n_loc: int):
    out = np.zeros(n_sku, np.int32)
    _check(_load().gen_slot_random(seed, n_sku, n_loc, _p(out)), "gen_slot_random")
    return out


def gen_slot_abc(seed: int, layout: Layout, n_sku: int, swap_frac: float):
    out = np.zeros(n_sku, np.int32)
    _check(_load().gen_slot_abc(seed, layout.n_aisles, layout.slots_per_side, layout.aisle_pitch,
                                layout.slot_pitch, layout.cross_aisle_width, n_sku, swap_frac, _p(out)),
           "gen_slot_abc")
    return out


def gen_plans(seed: int, mode: int, order_off: np.ndarray, n_plans: int, max_orders: int,
              max_lines: int = 0, plan_base: int = 0):
    lib = _load()
    n_orders = order_off.shape[0] - 1
    pto = np.zeros(n_plans + 1, np.int32)
    cap = max(1, n_plans * n_orders)
    to = np.zeros(cap + 1, np.int32)
    seq = np.zeros(max(1, n_plans * n_orders), np.int32)
    nt = _check(lib.gen_plans(seed, mode, _p(order_off), n_orders, n_plans, plan_base, max_orders,
                              max_lines, _p(pto), _p(to), _p(seq), cap), "gen_plans")
    return pto, np.ascontiguousarray(to[:nt + 1]), np.ascontiguousarray(seq[:n_plans * n_orders])


def gen_moves(seed: int, step: int, inst: Instance, moves_per_plan: int) -> np.ndarray:
    """int32 [n_plans, moves_per_plan, 4] moves {type, a, b, 0} (see gen.c)."""
    lib = _load()
    pool = np.ascontiguousarray(np.unique(inst.line_sku).astype(np.int32))
    ntours = np.ascontiguousarray(np.diff(inst.plan_tour_off).astype(np.int32))
    out = np.zeros((inst.n_plans, moves_per_plan, 4), np.int32)
    _check(lib.gen_moves(seed, step, inst.n_plans, moves_per_plan, inst.n_orders, _p(ntours), _p(pool),
                         pool.shape[0], inst.n_sku, _p(out)), "gen_moves")
    return out


def gen_relocations(seed: int, step: int, inst: Instance, moves_per_plan: int) -> np.ndarray:
    """int32 [n_plans, moves_per_plan, 4] relocation moves {3, sku, location,
    plan} (see gen.c)."""
    pool = np.ascontiguousarray(np.unique(inst.line_sku).astype(np.int32))
    out = np.zeros((inst.n_plans, moves_per_plan, 4), np.int32)
    _check(_load().gen_relocations(seed, step, inst.n_plans, moves_per_plan, _p(pool), pool.shape[0],
                                   inst.layout.n_loc, _p(out)), "gen_relocations")
    return out


def instance_param(seed: int, inst: int, which: int, lo: int, hi: int) -> int:
    return int(_load().gen_instance_param(seed, inst, which, lo, hi))


def stream_word(seed: int, tag: int, idx: int, n: int = 0) -> int:
    return int(_load().gen_stream_word(seed, tag, idx, n))


# ------------------------------------------------------------------------ presets

def tiny(seed: int = 1, n_plans: int = 64, plan_base: int = 0) -> Instance:
    """10 aisles x 30 slots/side (600 locations), 600 SKUs slotted by a random
    permutation, 200 orders of 1..5 distinct uniform SKUs (P(k) ~ 0.5^k),
    plans = random order sequence cut into chunks of 1..8 orders."""
    lay = Layout(10, 30)
    off, lines = gen_orders(seed, 200, 600, 5, 0.5, 0.0)
    slot = gen_slot_random(seed, 600, lay.n_loc)
    pto, to, seq = gen_plans(seed, 0, off, n_plans, 8, 0, plan_base)
    return Instance(lay, 600, off, lines, slot, pto, to, seq, {"name": "tiny", "seed": seed})


def midsize(seed: int = 2, n_plans: int = 4096, plan_base: int = 0) -> Instance:
    """40 aisles x 100 slots/side (8,000 locations), 8,000 SKUs with Zipf(1.1)
    popularity slotted ABC with 10% of slots swapped, 4,000 orders of 1..12
    lines (truncated geometric p=0.4, SKUs by popularity), plans greedily cut
    into tours of at most 20 orders / 60 lines."""
    lay = Layout(40, 100)
    off, lines = gen_orders(seed, 4000, 8000, 12, 0.4, 1.1)
    slot = gen_slot_abc(seed, lay, 8000, 0.10)
    pto, to, seq = gen_plans(seed, 1, off, n_plans, 20, 60, plan_base)
    return Instance(lay, 8000, off, lines, slot, pto, to, seq, {"name": "midsize", "seed": seed})


def batched_instance(seed: int, i: int, n_plans: int = 256) -> Instance:
    """Instance i of the uneven batch: aisles U[8,64], slots/side U[20,200],
    orders U[100,5000], n_sku = n_loc, other laws as ``midsize``."""
    a = instance_param(seed, i, 0, 8, 64)
    L = instance_param(seed, i, 1, 20, 200)
    n_orders = instance_param(seed, i, 2, 100, 5000)
    lay = Layout(a, L)
    n_sku = lay.n_loc
    iseed = (seed * 1_000_003 + i * 7919 + 17) & 0xFFFFFFFFFFFFFFFF
    off, lines = gen_orders(iseed, n_orders, n_sku, 12, 0.4, 1.1)
    slot = gen_slot_abc(iseed, lay, n_sku, 0.10)
    pto, to, seq = gen_plans(iseed, 1, off, n_plans, 20, 60)
    return Instance(lay, n_sku, off, lines, slot, pto, to, seq,
                    {"name": "batched", "seed": seed, "index": i})


def paperscale(seed: int = 4, n_plans: int = 16384, plan_base: int = 0) -> Instance:
    """500 aisles x 200 slots/side (200,000 locations), 50,000 SKUs Zipf(1.0)
    slotted ABC over the 50,000 nearest locations with 10% swapped, 4,000
    orders (~10,000 lines), tours of at most 24 orders (no line cap)."""
    lay = Layout(500, 200)
    off, lines = gen_orders(seed, 4000, 50000, 12, 0.4, 1.0)
    slot = gen_slot_abc(seed, lay, 50000, 0.10)
    pto, to, seq = gen_plans(seed, 1, off, n_plans, 24, 0, plan_base)
    return Instance(lay, 50000, off, lines, slot, pto, to, seq, {"name": "paperscale", "seed": seed})


def midsize_cat(seed: int = 6, n_plans: int = 256, plan_base: int = 0) -> Instance:
    """The mid-size layout and catalogue with a category structure: 8,000 SKUs
    in 64 categories (s mod 64), Zipf(1.1) popularity, 4,000 orders of 1..12
    lines of which 80 % come from the order's category; ABC slotting with 10 %
    swapped; plans as ``midsize``."""
    lay = Layout(40, 100)
    off, lines = gen_orders_cat(seed, 4000, 8000, 12, 0.4, 1.1, 64, 0.8)
    slot = gen_slot_abc(seed, lay, 8000, 0.10)
    pto, to, seq = gen_plans(seed, 1, off, n_plans, 20, 60, plan_base)
    return Instance(lay, 8000, off, lines, slot, pto, to, seq, {"name": "midsize_cat", "seed": seed})


def paperscale_cat(seed: int = 7, n_plans: int = 256, plan_base: int = 0) -> Instance:
    """The paper-scale layout (500 x 200, 200,000 locations) with 50,000 SKUs
    in 256 categories, Zipf(1.0), 4,000 orders of which 80 % of the lines come
    from the order's category; ABC slotting with 10 % swapped; tours of at
    most 24 orders."""
    lay = Layout(500, 200)
    off, lines = gen_orders_cat(seed, 4000, 50000, 12, 0.4, 1.0, 256, 0.8)
    slot = gen_slot_abc(seed, lay, 50000, 0.10)
    pto, to, seq = gen_plans(seed, 1, off, n_plans, 24, 0, plan_base)
    return Instance(lay, 50000, off, lines, slot, pto, to, seq, {"name": "paperscale_cat", "seed": seed})


PRESETS = {"tiny": tiny, "midsize": midsize, "paperscale": paperscale, "midsize_cat": midsize_cat,
           "paperscale_cat": paperscale_cat}
