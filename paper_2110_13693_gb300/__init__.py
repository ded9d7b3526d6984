"""GB300 warehouse order-picking plan evaluator -- Python binding.

A thin ctypes layer over ``libwh.so`` whose C ABI is ``include/wh.h``.  The
functions named ``wh_*`` mirror the C entry points one to one and only
marshal arguments; every step of the evaluation runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libwh.so")
_lib = None

WH_OK, WH_EINVAL, WH_ERANGE, WH_ENOMEM, WH_ECUDA, WH_ETIMEOUT = 0, -1, -2, -3, -4, -5
WH_ROUTE_SSHAPE, WH_ROUTE_OPTIMAL = 1, 2
WH_STATUS_BAD_ORDER, WH_STATUS_BAD_SKU, WH_STATUS_BAD_LOC = 1, 2, 4
WH_STATUS_BAD_OFFSET, WH_STATUS_TOUR_TOO_LONG, WH_STATUS_LONG_OVERFLOW = 8, 16, 32
WH_STATUS_TIMEOUT = 64
WH_NOALLOC_MAX_LINES, WH_NOALLOC_MAX_TOURS = 1 << 20, 1 << 20
ERRORS = {WH_EINVAL: "WH_EINVAL", WH_ERANGE: "WH_ERANGE", WH_ENOMEM: "WH_ENOMEM",
          WH_ECUDA: "WH_ECUDA", WH_ETIMEOUT: "WH_ETIMEOUT"}


class WhError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {ERRORS.get(code, code)}")
        self.code = code


class wh_layout_desc(ctypes.Structure):
    _fields_ = [("n_aisles", ctypes.c_int32), ("slots_per_side", ctypes.c_int32),
                ("aisle_pitch", ctypes.c_int32), ("slot_pitch", ctypes.c_int32),
                ("cross_aisle_width", ctypes.c_int32)]


class wh_orders(ctypes.Structure):
    _fields_ = [("n_orders", ctypes.c_int32), ("n_lines", ctypes.c_int32), ("n_sku", ctypes.c_int32),
                ("order_off", ctypes.c_void_p), ("line_sku", ctypes.c_void_p)]


class wh_plans(ctypes.Structure):
    _fields_ = [("n_plans", ctypes.c_int32), ("n_tours", ctypes.c_int32), ("n_seq", ctypes.c_int64),
                ("slot_map", ctypes.c_void_p), ("slot_map_stride", ctypes.c_int64),
                ("plan_tour_off", ctypes.c_void_p), ("tour_off", ctypes.c_void_p),
                ("order_seq", ctypes.c_void_p), ("loc_used", ctypes.c_void_p)]


class wh_costs(ctypes.Structure):
    _fields_ = [("tour_s", ctypes.c_void_p), ("tour_rr", ctypes.c_void_p),
                ("plan_s", ctypes.c_void_p), ("plan_rr", ctypes.c_void_p)]


class wh_instance(ctypes.Structure):
    _fields_ = [("layout", wh_layout_desc), ("orders", wh_orders), ("plans", wh_plans), ("out", wh_costs),
                ("order_seq16", ctypes.c_void_p)]


# every symbol include/wh.h declares, with its ctypes signature
SIGNATURES = {
    "wh_create_layout": (ctypes.c_int, [ctypes.POINTER(wh_layout_desc), ctypes.POINTER(ctypes.c_void_p)]),
    "wh_eval_plans": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(wh_orders), ctypes.POINTER(wh_plans),
                                     ctypes.c_uint32, ctypes.POINTER(wh_costs), ctypes.c_void_p]),
    "wh_get_last_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]),
    "wh_ls_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(wh_orders), ctypes.POINTER(wh_plans),
                                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "wh_eval_moves": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(wh_orders), ctypes.POINTER(wh_plans),
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "wh_eval_plans_noalloc": (ctypes.c_int, [ctypes.POINTER(wh_layout_desc), ctypes.POINTER(wh_orders),
                                             ctypes.POINTER(wh_plans), ctypes.c_uint32,
                                             ctypes.POINTER(wh_costs), ctypes.c_void_p, ctypes.c_void_p]),
    "wh_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "wh_get_move_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int64)]),
    "wh_get_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_int32]),
    "wh_destroy": (None, [ctypes.c_void_p]),
    "wh_batch_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "wh_batch_get_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int32]),
    "wh_batch_create": (ctypes.c_int, [ctypes.POINTER(wh_instance), ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "wh_batch_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "wh_batch_get_tuning": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int32)] * 3),
    "wh_batch_eval": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "wh_batch_eval_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "wh_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_char_p, ctypes.c_void_p]
                          + [ctypes.POINTER(ctypes.c_int32)] * 3),
    "wh_batch_get_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]),
    "wh_batch_destroy": (None, [ctypes.c_void_p]),
    "wh_surrogate_features": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(wh_orders), ctypes.POINTER(wh_plans),
                                             ctypes.c_void_p, ctypes.c_void_p]),
    "wh_surrogate_create": (ctypes.c_int, [ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)]),
    "wh_surrogate_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "wh_surrogate_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                               ctypes.POINTER(ctypes.c_float)]),
    "wh_surrogate_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "wh_surrogate_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                               ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "wh_surrogate_screen": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(wh_orders),
                                           ctypes.POINTER(wh_plans), ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "wh_surrogate_screen_eval": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(wh_orders),
                                                ctypes.POINTER(wh_plans), ctypes.c_void_p, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "wh_surrogate_screen_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                                 ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                                 ctypes.POINTER(ctypes.c_void_p)]),
    "wh_surrogate_get_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint32)]),
    "wh_surrogate_predict_timeout_test": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                         ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                                         ctypes.c_void_p]),
    "wh_surrogate_get_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.c_void_p]),
    "wh_batch_grow": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(wh_orders), ctypes.c_void_p, ctypes.c_int64,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "wh_widen_u16": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "wh_occupancy": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(wh_orders), ctypes.POINTER(wh_plans),
                                    ctypes.c_void_p]),
    "wh_kmeans_slotting": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(wh_orders), ctypes.c_void_p,
                                          ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "wh_routes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(wh_orders), ctypes.POINTER(wh_plans),
                                 ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p]),
    "wh_surrogate_destroy": (None, [ctypes.c_void_p]),
}
WH_MLP_NPARAM, WH_FEATURES = 115457, 192
(WH_TRACE_Z1, WH_TRACE_H1, WH_TRACE_Z2, WH_TRACE_H2, WH_TRACE_Y, WH_TRACE_DY, WH_TRACE_DZ2,
 WH_TRACE_DZ1) = range(8)


def library_path() -> str:
    return _SO


def load():
    """Load libwh.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            raise RuntimeError(f"CUDA library {_SO} is missing: run __graft_entry__.build() first")
        lib = ctypes.CDLL(_SO)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int, what: str) -> None:
    if rc != WH_OK:
        raise WhError(rc, what)


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


# ------------------------------------------------------------- C entry points

def wh_create_layout(n_aisles: int, slots_per_side: int, aisle_pitch: int = 3, slot_pitch: int = 1,
                     cross_aisle_width: int = 2) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    desc = wh_layout_desc(n_aisles, slots_per_side, aisle_pitch, slot_pitch, cross_aisle_width)
    _check(load().wh_create_layout(ctypes.byref(desc), ctypes.byref(h)), "wh_create_layout")
    return h


def wh_eval_plans(layout, orders: wh_orders, plans: wh_plans, routing_mask: int, out: wh_costs,
                  stream=None) -> None:
    _check(load().wh_eval_plans(layout, ctypes.byref(orders), ctypes.byref(plans), routing_mask,
                                ctypes.byref(out), _stream_ptr(stream)), "wh_eval_plans")


def wh_eval_plans_noalloc(desc: wh_layout_desc, orders: wh_orders, plans: wh_plans, routing_mask: int,
                          out: wh_costs, status_ptr: int = 0, stream=None) -> None:
    """Same results as wh_eval_plans, for callers that cannot allocate device
    memory: scratch comes from a fixed array inside the library (limits
    WH_NOALLOC_MAX_LINES / WH_NOALLOC_MAX_TOURS); concurrent calls race."""
    _check(load().wh_eval_plans_noalloc(ctypes.byref(desc), ctypes.byref(orders), ctypes.byref(plans),
                                        routing_mask, ctypes.byref(out), ctypes.c_void_p(status_ptr or None),
                                        _stream_ptr(stream)), "wh_eval_plans_noalloc")


def wh_eval_moves(layout, orders: wh_orders, plans: wh_plans, tour_s, tour_rr, moves, n_moves: int,
                  max_orders: int, max_lines: int, delta, status, stream=None) -> None:
    """Pointers (ints) for tour_s, tour_rr, moves, delta and status."""
    _check(load().wh_eval_moves(layout, ctypes.byref(orders), ctypes.byref(plans), ctypes.c_void_p(tour_s),
                                ctypes.c_void_p(tour_rr), ctypes.c_void_p(moves), n_moves, max_orders, max_lines,
                                ctypes.c_void_p(delta), ctypes.c_void_p(status), _stream_ptr(stream)),
           "wh_eval_moves")


def wh_ls_apply(layout, orders: wh_orders, plans: wh_plans, moves, moves_per_plan: int, delta, status, applied,
                costs=None, tour_changed=None, stream=None) -> None:
    """costs: a wh_costs to update in place (or None); tour_changed: device
    pointer of a uint8 per tour, set for every rewritten tour (or None)."""
    _check(load().wh_ls_apply(layout, ctypes.byref(orders), ctypes.byref(plans), ctypes.c_void_p(moves),
                              moves_per_plan, ctypes.c_void_p(delta), ctypes.c_void_p(status),
                              ctypes.c_void_p(applied), ctypes.byref(costs) if costs is not None else None,
                              ctypes.c_void_p(tour_changed), _stream_ptr(stream)), "wh_ls_apply")


def wh_get_last_status(layout, stream=None) -> int:
    v = ctypes.c_uint32(0)
    _check(load().wh_get_last_status(layout, _stream_ptr(stream), ctypes.byref(v)), "wh_get_last_status")
    return int(v.value)


def wh_get_move_stats(layout, stream=None):
    """(changed tours walked, their lines) of the last wh_eval_moves call."""
    t, l = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().wh_get_move_stats(layout, _stream_ptr(stream), ctypes.byref(t), ctypes.byref(l)),
           "wh_get_move_stats")
    return int(t.value), int(l.value)


def wh_set_timing(layout, enable: bool) -> None:
    _check(load().wh_set_timing(layout, 1 if enable else 0), "wh_set_timing")


def wh_get_timing(layout) -> dict:
    """{kernel name: (launches, total ms)} since timing was enabled."""
    cap = 16
    n = ctypes.c_int32(0)
    names = (ctypes.c_char_p * cap)()
    launches = (ctypes.c_int32 * cap)()
    ms = (ctypes.c_double * cap)()
    _check(load().wh_get_timing(layout, ctypes.byref(n), names, launches, ms, cap), "wh_get_timing")
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(n.value, cap))}


def wh_batch_set_timing(batch, enable: bool) -> None:
    _check(load().wh_batch_set_timing(batch, 1 if enable else 0), "wh_batch_set_timing")


def wh_batch_get_timing(batch) -> dict:
    """{kernel name: (launches, total ms)} of the batch's eager launches since
    timing was enabled."""
    cap = 16
    n = ctypes.c_int32(0)
    names = (ctypes.c_char_p * cap)()
    launches = (ctypes.c_int32 * cap)()
    ms = (ctypes.c_double * cap)()
    _check(load().wh_batch_get_timing(batch, ctypes.byref(n), names, launches, ms, cap), "wh_batch_get_timing")
    return {names[i].decode(): (int(launches[i]), float(ms[i])) for i in range(min(n.value, cap))}


def wh_destroy(layout) -> None:
    load().wh_destroy(layout)


def wh_batch_create(instances) -> ctypes.c_void_p:
    arr = (wh_instance * len(instances))(*instances)
    h = ctypes.c_void_p()
    _check(load().wh_batch_create(arr, len(instances), ctypes.byref(h)), "wh_batch_create")
    return h


def wh_batch_set_tuning(batch, threads: int, chunks_per_item: int, smem_tables: int = 1) -> None:
    _check(load().wh_batch_set_tuning(batch, threads, chunks_per_item, smem_tables), "wh_batch_set_tuning")


def wh_batch_get_tuning(batch):
    v = [ctypes.c_int32() for _ in range(3)]
    _check(load().wh_batch_get_tuning(batch, *[ctypes.byref(x) for x in v]), "wh_batch_get_tuning")
    return tuple(int(x.value) for x in v)


def wh_batch_eval(batch, routing_mask: int, stream=None) -> None:
    _check(load().wh_batch_eval(batch, routing_mask, _stream_ptr(stream)), "wh_batch_eval")


def wh_batch_eval_graph(batch, routing_mask: int, stream=None) -> None:
    _check(load().wh_batch_eval_graph(batch, routing_mask, _stream_ptr(stream)), "wh_batch_eval_graph")


def wh_batch_autotune(batch, routing_mask: int, cache_path=None, stream=None):
    """Returns (threads, chunks_per_item, from_cache)."""
    v = [ctypes.c_int32() for _ in range(3)]
    path = None if cache_path is None else os.fsencode(cache_path)
    _check(load().wh_batch_autotune(batch, routing_mask, path, _stream_ptr(stream), *[ctypes.byref(x) for x in v]),
           "wh_batch_autotune")
    return tuple(int(x.value) for x in v)


def wh_batch_get_status(batch, stream=None) -> int:
    v = ctypes.c_uint32(0)
    _check(load().wh_batch_get_status(batch, _stream_ptr(stream), ctypes.byref(v)), "wh_batch_get_status")
    return int(v.value)


def wh_batch_destroy(batch) -> None:
    load().wh_batch_destroy(batch)


# ------------------------------------------------------ tensor-level helpers

def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


@dataclass
class DeviceProblem:
    """Orders and plans resident on one device (int32 tensors) plus the
    ctypes views the C calls take.  Keeps the tensors alive."""
    order_off: object
    line_sku: object
    slot_map: object
    plan_tour_off: object
    tour_off: object
    order_seq: object
    n_sku: int
    slot_map_stride: int = 0
    loc_used: object = None     # per-plan occupancy bits (relocation moves), see occupancy()
    order_seq16: object = None  # the order ids as 16-bit values (batched instances; order_seq may be None)

    @property
    def n_plans(self) -> int:
        return int(self.plan_tour_off.shape[0] - 1)

    @property
    def n_tours(self) -> int:
        return int(self.tour_off.shape[0] - 1)

    def orders(self) -> wh_orders:
        return wh_orders(int(self.order_off.shape[0] - 1), int(self.line_sku.shape[0]), self.n_sku,
                         _ptr(self.order_off), _ptr(self.line_sku))

    def plans(self) -> wh_plans:
        seq = self.order_seq if self.order_seq is not None else self.order_seq16
        return wh_plans(self.n_plans, self.n_tours, int(seq.shape[0]), _ptr(self.slot_map),
                        self.slot_map_stride, _ptr(self.plan_tour_off), _ptr(self.tour_off),
                        _ptr(self.order_seq), _ptr(self.loc_used))


def to_device(inst, device="cuda", slot_map=None, slot_map_stride: int = 0) -> DeviceProblem:
    """Copy a generated instance (numpy CSR arrays) to `device`."""
    import torch

    def t(a):
        return torch.as_tensor(a, dtype=torch.int32).to(device).contiguous()

    smap = inst.slot_map if slot_map is None else slot_map
    return DeviceProblem(t(inst.order_off), t(inst.line_sku), t(smap), t(inst.plan_tour_off),
                         t(inst.tour_off), t(inst.order_seq), int(inst.n_sku), int(slot_map_stride))


@dataclass
class Costs:
    tour_s: object
    tour_rr: object
    plan_s: object
    plan_rr: object

    def c(self) -> wh_costs:
        return wh_costs(_ptr(self.tour_s), _ptr(self.tour_rr), _ptr(self.plan_s), _ptr(self.plan_rr))


def alloc_costs(n_tours: int, n_plans: int, device="cuda", tours: bool = True) -> Costs:
    import torch
    ti = (lambda: torch.empty(max(n_tours, 1), dtype=torch.int32, device=device)) if tours else (lambda: None)
    return Costs(ti(), ti(), torch.empty(max(n_plans, 1), dtype=torch.int64, device=device),
                 torch.empty(max(n_plans, 1), dtype=torch.int64, device=device))


class Layout:
    """Owning wrapper of a ``wh_layout`` handle."""

    def __init__(self, n_aisles, slots_per_side, aisle_pitch=3, slot_pitch=1, cross_aisle_width=2):
        self.desc = (n_aisles, slots_per_side, aisle_pitch, slot_pitch, cross_aisle_width)
        self.handle = wh_create_layout(*self.desc)

    @classmethod
    def of(cls, lay) -> "Layout":
        return cls(lay.n_aisles, lay.slots_per_side, lay.aisle_pitch, lay.slot_pitch, lay.cross_aisle_width)

    def eval_plans(self, prob: DeviceProblem, costs: Costs, mask: int = 3, stream=None) -> Costs:
        wh_eval_plans(self.handle, prob.orders(), prob.plans(), mask, costs.c(), stream)
        return costs

    def status(self, stream=None) -> int:
        return wh_get_last_status(self.handle, stream)

    def eval_moves(self, prob: DeviceProblem, costs: Costs, moves, max_orders: int = 0, max_lines: int = 0,
                   stream=None):
        """Deltas [n, 2] int64 and status [n] int32 (device tensors) of moves
        ([n, 4] int32 device tensor) against the current costs `costs`."""
        import torch
        mv = moves.reshape(-1, 4).contiguous()
        n = int(mv.shape[0])
        delta = torch.empty((max(n, 1), 2), dtype=torch.int64, device=mv.device)
        status = torch.empty(max(n, 1), dtype=torch.int32, device=mv.device)
        wh_eval_moves(self.handle, prob.orders(), prob.plans(), _ptr(costs.tour_s), _ptr(costs.tour_rr),
                      _ptr(mv), n, max_orders, max_lines, _ptr(delta), _ptr(status), stream)
        return delta[:n], status[:n]

    def ls_step(self, prob: DeviceProblem, costs: Costs, moves, moves_per_plan: int, max_orders: int = 0,
                max_lines: int = 0, stream=None, refresh: bool = False, changed=None):
        """One exact local-search step: score the moves, apply each plan's best
        improving move in place and update the costs of the changed tours
        (refresh=True re-scores every tour instead).  `changed` (uint8 device
        tensor, one byte per tour) gets a 1 for every rewritten tour.  Returns
        applied [n_plans]."""
        import torch
        mv = moves.reshape(-1, 4).contiguous()
        delta, status = self.eval_moves(prob, costs, mv, max_orders, max_lines, stream)
        applied = torch.empty(max(prob.n_plans, 1), dtype=torch.int32, device=mv.device)
        wh_ls_apply(self.handle, prob.orders(), prob.plans(), _ptr(mv), moves_per_plan, _ptr(delta), _ptr(status),
                    _ptr(applied), None if refresh else costs.c(), None if changed is None else _ptr(changed), stream)
        if refresh:
            self.eval_plans(prob, costs, 3, stream)
        return applied[:prob.n_plans]

    def screen(self, surrogate: "Surrogate", prob: DeviceProblem, moves, moves_per_plan: int, keep: int,
               max_orders: int = 0, max_lines: int = 0, stream=None, y_tour=None, changed=None):
        """The `keep` most promising moves per plan by the surrogate's
        prediction: int32 [n_plans * keep, 4] (device).  With y_tour (float32
        per tour) the current tours' predictions are kept there between
        calls: with `changed` (uint8 per tour, as ls_step sets it) only the
        flagged tours are re-predicted and their flags cleared, without it
        every tour is."""
        import torch
        mv = moves.reshape(-1, 4).contiguous()
        kept = torch.empty((max(prob.n_plans * keep, 1), 4), dtype=torch.int32, device=mv.device)
        wh_surrogate_screen(self.handle, surrogate.handle, prob.orders(), prob.plans(), _ptr(mv), moves_per_plan,
                            keep, max_orders, max_lines, _ptr(kept), None if y_tour is None else _ptr(y_tour),
                            None if changed is None else _ptr(changed), stream)
        return kept[:prob.n_plans * keep]

    def screen_eval(self, surrogate: "Surrogate", prob: DeviceProblem, costs: Costs, moves, moves_per_plan: int,
                    keep: int, max_orders: int = 0, max_lines: int = 0, stream=None, y_tour=None, changed=None):
        """screen() and the exact scores of the kept moves in one call:
        (kept int32 [n_plans * keep, 4], delta int64 [n, 2], status int32 [n]),
        the scores as eval_moves(kept) gives them; pass them to apply_scored."""
        import torch
        mv = moves.reshape(-1, 4).contiguous()
        n = max(prob.n_plans * keep, 1)
        kept = torch.empty((n, 4), dtype=torch.int32, device=mv.device)
        delta = torch.empty((n, 2), dtype=torch.int64, device=mv.device)
        status = torch.empty(n, dtype=torch.int32, device=mv.device)
        wh_surrogate_screen_eval(self.handle, surrogate.handle, prob.orders(), prob.plans(), _ptr(mv), moves_per_plan,
                                 keep, max_orders, max_lines, None if y_tour is None else _ptr(y_tour),
                                 None if changed is None else _ptr(changed), _ptr(costs.tour_s), _ptr(costs.tour_rr),
                                 _ptr(kept), _ptr(delta), _ptr(status), stream)
        k = prob.n_plans * keep
        return kept[:k], delta[:k], status[:k]

    def apply_scored(self, prob: DeviceProblem, costs: Costs, moves, moves_per_plan: int, delta, status,
                     stream=None, changed=None):
        """Apply each plan's best improving move of `moves` scored by the last
        move evaluation on this layout (eval_moves or screen_eval of exactly
        these moves), costs updated incrementally.  Returns applied [n_plans]."""
        import torch
        applied = torch.empty(max(prob.n_plans, 1), dtype=torch.int32, device=moves.device)
        wh_ls_apply(self.handle, prob.orders(), prob.plans(), _ptr(moves), moves_per_plan, _ptr(delta), _ptr(status),
                    _ptr(applied), costs.c(), None if changed is None else _ptr(changed), stream)
        return applied[:prob.n_plans]

    def screen_trace(self):
        """The last screen's tasks (int32 [n, 4]: move, changed tour, two
        move-specific ids), counted flags (int32 [n, 2]) and feature rows
        (bf16 [n, 192]), copied to torch tensors; None after any other call."""
        import torch
        n, t, c, f = wh_surrogate_screen_trace(self.handle)
        if n == 0 or not t:
            return None
        tasks = torch.as_tensor(_DeviceView(t, (n, 4), "<i4"), device="cuda").clone()
        counted = torch.as_tensor(_DeviceView(c, (n, 2), "<i4"), device="cuda").clone()
        rows = torch.as_tensor(_DeviceView(f, (n, WH_FEATURES), "<i2"), device="cuda").clone().view(torch.bfloat16)
        return tasks, counted, rows

    def batch_grow(self, prob: DeviceProblem, slot_maps, max_orders: int, max_lines: int = 0, stream=None):
        """Seed-and-grow batching of prob's orders under each slotting of
        slot_maps (int32 device, [n_maps, n_sku] or [n_sku]): returns
        (tour_off [n_maps, n_orders + 1], order_seq [n_maps, n_orders],
        n_tours [n_maps]) device tensors (valid tour_off entries: n_tours + 1)."""
        import torch
        maps = slot_maps.reshape(-1, prob.n_sku).contiguous()
        n_maps = int(maps.shape[0])
        n_orders = int(prob.order_off.numel()) - 1
        dev = maps.device
        tour_off = torch.zeros((n_maps, n_orders + 1), dtype=torch.int32, device=dev)
        order_seq = torch.zeros((n_maps, max(n_orders, 1)), dtype=torch.int32, device=dev)
        n_tours = torch.zeros(n_maps, dtype=torch.int32, device=dev)
        wh_batch_grow(self.handle, prob.orders(), _ptr(maps), prob.n_sku, n_maps, max_orders, max_lines,
                      _ptr(tour_off), _ptr(order_seq), _ptr(n_tours), stream)
        return tour_off, order_seq[:, :n_orders], n_tours

    def occupancy(self, prob: DeviceProblem, stream=None):
        """Build prob.loc_used (per-plan occupancy bits, int32 device tensor)
        from prob's per-plan slottings, for relocation moves; returns it."""
        import torch
        words = (self.desc[0] * 2 * self.desc[1] + 31) // 32
        if prob.loc_used is None or prob.loc_used.numel() != prob.n_plans * words:
            prob.loc_used = torch.zeros(max(prob.n_plans * words, 1), dtype=torch.int32,
                                        device=prob.order_off.device)
        _check(load().wh_occupancy(self.handle, ctypes.byref(prob.orders()), ctypes.byref(prob.plans()),
                                   _stream_ptr(stream)), "wh_occupancy")
        return prob.loc_used

    def kmeans_slotting(self, prob: DeviceProblem, signs, k: int, iters: int, freq_weight: int = 64, init=None,
                        u=None, stream=None):
        """K-means slotting of prob's SKUs (see wh_kmeans_slotting): signs int8
        [n_sku, 32] of +-1 and either init (int32 [k] SKU ids) or u (the k
        uint64 K-means++ draws, held as the bits of an int64 tensor), device
        tensors.  Returns (x [n_sku, 32], seeds [k], centroids [k, 32], assign
        [n_sku], slot_map [n_sku]) device tensors."""
        import torch
        dev = prob.order_off.device
        n_sku = prob.n_sku
        sg = signs.reshape(n_sku, 32).to(torch.int8).contiguous()
        x = torch.empty((n_sku, 32), dtype=torch.int32, device=dev)
        seeds = torch.empty(k, dtype=torch.int32, device=dev)
        cent = torch.empty((k, 32), dtype=torch.int32, device=dev)
        assign = torch.empty(n_sku, dtype=torch.int32, device=dev)
        smap = torch.empty(n_sku, dtype=torch.int32, device=dev)
        ini = None if init is None else init.to(torch.int32).contiguous()
        uu = None if u is None else u.contiguous()
        wh_kmeans_slotting(self.handle, prob.orders(), _ptr(sg), freq_weight, k,
                           None if ini is None else _ptr(ini), None if uu is None else _ptr(uu), iters, _ptr(x),
                           _ptr(seeds), _ptr(cent), _ptr(assign), _ptr(smap), stream)
        return x, seeds, cent, assign, smap

    def routes(self, prob: DeviceProblem, tours, max_points: int = 256, stream=None):
        """Optimal pick sequences of the listed tours (int32 device tensor of
        global tour indices): (points [n, max_points] int32, aisle << 16 |
        slot in visiting order, n_points [n], length [n]) device tensors."""
        import torch
        tl = tours.reshape(-1).to(torch.int32).contiguous()
        n = int(tl.numel())
        dev = tl.device
        points = torch.full((max(n, 1), max(max_points, 1)), -1, dtype=torch.int32, device=dev)
        n_points = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        length = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        wh_routes(self.handle, prob.orders(), prob.plans(), _ptr(tl), n, max_points, _ptr(points), _ptr(n_points),
                  _ptr(length), stream)
        return points[:n, :max_points], n_points[:n], length[:n]

    def set_timing(self, enable: bool) -> None:
        wh_set_timing(self.handle, enable)

    def timing(self) -> dict:
        return wh_get_timing(self.handle)

    def move_stats(self, stream=None):
        return wh_get_move_stats(self.handle, stream)

    def close(self):
        if self.handle is not None and self.handle.value:
            wh_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def evaluate(layout: Layout, prob: DeviceProblem, mask: int = 3, tours: bool = True, stream=None) -> Costs:
    """Allocate outputs and score every tour and plan of `prob`."""
    costs = alloc_costs(prob.n_tours, prob.n_plans, prob.order_off.device, tours)
    return layout.eval_plans(prob, costs, mask, stream)


def evaluate_host(layout: Layout, host: DeviceProblem, dev: DeviceProblem, costs: Costs,
                  host_plan_out, mask: int = 3, stream=None):
    """End-to-end call from host memory: copy the pinned host inputs of `host`
    into the device buffers of `dev` (same shapes), evaluate, and copy the
    per-plan costs back into the pinned `host_plan_out` ([2, n_plans] int64).
    Returns (bytes host->device, bytes device->host)."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    h2d = 0
    with torch.cuda.stream(s):
        for name in ("order_off", "line_sku", "slot_map", "plan_tour_off", "tour_off", "order_seq"):
            src, dst = getattr(host, name), getattr(dev, name)
            dst.copy_(src, non_blocking=True)
            h2d += src.numel() * src.element_size()
        layout.eval_plans(dev, costs, mask, s)
        host_plan_out[0].copy_(costs.plan_s[:dev.n_plans], non_blocking=True)
        host_plan_out[1].copy_(costs.plan_rr[:dev.n_plans], non_blocking=True)
    d2h = 2 * dev.n_plans * 8
    return h2d, d2h


class HostPipeline:
    """End-to-end scoring of host-resident plan batches (pinned memory) with
    the host->device copy of one batch overlapping the evaluation of the
    previous one: two device buffer sets (DeviceProblem + Costs, shaped like
    the batches), a copy stream and a compute stream ordered by CUDA events.
    Every submitted batch has all its inputs copied in and its per-plan costs
    copied back; wait(ticket) returns once that batch's costs are on the host."""

    def __init__(self, layout: "Layout", bufs, mask: int = 3):
        import torch
        self.layout, self.bufs, self.mask = layout, list(bufs), mask
        self.copy, self.compute = torch.cuda.Stream(), torch.cuda.Stream()
        self.copied = [torch.cuda.Event() for _ in self.bufs]
        self.done = [torch.cuda.Event() for _ in self.bufs]
        self.stage16 = [None for _ in self.bufs]      # device landing buffers of 16-bit order ids
        self.k = 0

    def submit(self, host: DeviceProblem, host_plan_out):
        """Enqueue one batch; returns (ticket, bytes host->device, bytes device->host).
        host.order_seq may be int16 (order ids as unsigned 16-bit values, for
        n_orders <= 65,536): it crosses the link at 2 bytes per id and is
        widened on the device (wh_widen_u16) into the slot's int32 buffer."""
        import torch
        slot = self.k % len(self.bufs)
        self.k += 1
        dev, costs = self.bufs[slot]
        h2d = 0
        self.copy.wait_event(self.done[slot])          # the buffer's previous batch is finished
        with torch.cuda.stream(self.copy):
            for name in ("order_off", "line_sku", "slot_map", "plan_tour_off", "tour_off", "order_seq"):
                src, dst = getattr(host, name), getattr(dev, name)
                if name == "order_seq" and src.dtype == torch.int16:
                    st = self.stage16[slot]
                    if st is None or st.numel() != src.numel():
                        st = self.stage16[slot] = torch.empty(src.numel(), dtype=torch.int16, device=dst.device)
                    st.copy_(src, non_blocking=True)
                    _check(load().wh_widen_u16(ctypes.c_void_p(_ptr(st)), ctypes.c_void_p(_ptr(dst)), src.numel(),
                                               _stream_ptr(self.copy)), "wh_widen_u16")
                else:
                    dst.copy_(src, non_blocking=True)
                h2d += src.numel() * src.element_size()
            self.copied[slot].record(self.copy)
        self.compute.wait_event(self.copied[slot])
        with torch.cuda.stream(self.compute):
            self.layout.eval_plans(dev, costs, self.mask, self.compute)
            host_plan_out[0].copy_(costs.plan_s[:dev.n_plans], non_blocking=True)
            host_plan_out[1].copy_(costs.plan_rr[:dev.n_plans], non_blocking=True)
            self.done[slot].record(self.compute)
        return slot, h2d, 2 * dev.n_plans * 8

    def wait(self, ticket) -> None:
        self.done[ticket].synchronize()


class Batch:
    """Owning wrapper of a ``wh_batch``: many instances (each a Layout
    geometry tuple, a DeviceProblem and its Costs) scored in one launch."""

    def __init__(self, items):
        self._keep = list(items)
        insts = []
        for desc, prob, costs in self._keep:
            insts.append(wh_instance(wh_layout_desc(*desc), prob.orders(), prob.plans(), costs.c(),
                                     _ptr(prob.order_seq16)))
        self.handle = wh_batch_create(insts)

    def eval(self, mask: int = 3, stream=None, graph: bool = False) -> None:
        (wh_batch_eval_graph if graph else wh_batch_eval)(self.handle, mask, stream)

    def set_tuning(self, threads: int, chunks_per_item: int, smem_tables: int = 1) -> None:
        wh_batch_set_tuning(self.handle, threads, chunks_per_item, smem_tables)

    def tuning(self):
        return wh_batch_get_tuning(self.handle)

    def autotune(self, mask: int = 3, cache_path=None, stream=None):
        return wh_batch_autotune(self.handle, mask, cache_path, stream)

    def status(self, stream=None) -> int:
        return wh_batch_get_status(self.handle, stream)

    def set_timing(self, enable: bool) -> None:
        wh_batch_set_timing(self.handle, enable)

    def timing(self) -> dict:
        return wh_batch_get_timing(self.handle)

    def close(self):
        if self.handle is not None and self.handle.value:
            wh_batch_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PackedInstances:
    """Many instances packed into two flat arrays, ready for one copy each
    across the host link: int32 ``flat`` holds, per instance, order_off,
    line_sku, slot_map, plan_tour_off and tour_off; ``seq16`` holds every
    instance's order ids as unsigned 16-bit values (each instance must have
    at most 65,536 orders).  Segments start on 16-byte boundaries (int32
    segments on multiples of 4 elements, the 16-bit order ids on multiples of
    8).  ``pin()`` moves
    both arrays to pinned host memory; ``device_set()`` makes a device copy
    with per-instance DeviceProblem / Costs views and a Batch over them."""

    FIELDS = ("order_off", "line_sku", "slot_map", "plan_tour_off", "tour_off")

    def __init__(self, insts):
        import numpy as np
        import torch
        self.geo, self.offsets, self.seq_off, self.n_sku = [], [], [], []
        self.n_tours, self.n_plans = [], []
        parts, seqs, pos, spos = [], [], 0, 0
        for inst in insts:
            if inst.n_orders > 65536:
                raise ValueError("16-bit order ids need at most 65,536 orders")
            lay = inst.layout
            self.geo.append((lay.n_aisles, lay.slots_per_side, lay.aisle_pitch, lay.slot_pitch,
                             lay.cross_aisle_width))
            offs = []
            for f in self.FIELDS:
                a = np.asarray(getattr(inst, f), np.int32)
                offs.append((pos, a.size))
                pad = (-a.size) % 4
                parts.append(a)
                if pad:
                    parts.append(np.zeros(pad, np.int32))
                pos += a.size + pad
            self.offsets.append(offs)
            q = np.asarray(inst.order_seq).astype(np.uint16)
            self.seq_off.append((spos, q.size))
            pad = (-q.size) % 8
            seqs.append(q)
            if pad:
                seqs.append(np.zeros(pad, np.uint16))
            spos += q.size + pad
            self.n_sku.append(int(inst.n_sku))
            self.n_tours.append(int(inst.n_tours))
            self.n_plans.append(int(inst.n_plans))
        self.flat = torch.from_numpy(np.concatenate(parts) if parts else np.zeros(4, np.int32))
        self.seq16 = torch.from_numpy((np.concatenate(seqs) if seqs else np.zeros(8, np.uint16)).view(np.int16))
        self.total_tours, self.total_plans = sum(self.n_tours), sum(self.n_plans)

    def pin(self) -> "PackedInstances":
        self.flat = self.flat.pin_memory()
        self.seq16 = self.seq16.pin_memory()
        return self

    @property
    def h2d_bytes(self) -> int:
        return self.flat.numel() * 4 + self.seq16.numel() * 2

    def device_set(self, device="cuda"):
        return PackedDeviceSet(self, device)


class PackedDeviceSet:
    """Device buffers shaped like a PackedInstances (flat int32 arrays, the
    16-bit order ids, per-instance outputs) and a Batch over per-instance
    views of them; the batch reads the 16-bit order ids directly.  The
    per-instance DeviceProblems carry no int32 order ids (order_seq None):
    they serve this batch only."""

    def __init__(self, packed: PackedInstances, device="cuda"):
        import torch
        self.packed = packed
        self.flat = torch.empty(packed.flat.numel(), dtype=torch.int32, device=device)
        self.seq16 = torch.empty(packed.seq16.numel(), dtype=torch.int16, device=device)
        self.tour_s = torch.empty(max(packed.total_tours, 1), dtype=torch.int32, device=device)
        self.tour_rr = torch.empty_like(self.tour_s)
        self.plan_s = torch.empty(max(packed.total_plans, 1), dtype=torch.int64, device=device)
        self.plan_rr = torch.empty_like(self.plan_s)
        items, t0, p0 = [], 0, 0
        for i, geo in enumerate(packed.geo):
            v = [self.flat[o:o + n] for o, n in packed.offsets[i]]
            so, sn = packed.seq_off[i]
            prob = DeviceProblem(v[0], v[1], v[2], v[3], v[4], None, packed.n_sku[i],
                                 order_seq16=self.seq16[so:so + sn])
            nt, npl = packed.n_tours[i], packed.n_plans[i]
            costs = Costs(self.tour_s[t0:t0 + nt], self.tour_rr[t0:t0 + nt], self.plan_s[p0:p0 + npl],
                          self.plan_rr[p0:p0 + npl])
            items.append((geo, prob, costs))
            t0 += nt
            p0 += npl
        self.items = items
        self.batch = Batch(items)

    def load(self, stream=None) -> None:
        """Copy the packed host arrays in (two copies), on `stream`."""
        import torch
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            self.flat.copy_(self.packed.flat, non_blocking=True)
            self.seq16.copy_(self.packed.seq16, non_blocking=True)

    def close(self):
        self.batch.close()


class PackedPipeline:
    """End-to-end batched scoring from pinned host memory: every submitted
    step copies all instances' inputs in (one copy of the int32 arrays, one
    of the 16-bit order ids, which the batch reads as they are), scores them in one
    persistent launch replayed as a CUDA graph, and copies every plan's two
    costs back to a pinned host array.  Two device sets alternate, so the
    copy of one step (copy stream) overlaps the evaluation of the previous
    one (compute stream)."""

    def __init__(self, packed: PackedInstances, mask: int = 3, tuning=None, slots: int = 2):
        import torch
        self.packed, self.mask = packed, mask
        self.sets = [PackedDeviceSet(packed) for _ in range(slots)]
        if tuning is not None:
            for d in self.sets:
                d.batch.set_tuning(*tuning)
        self.copy, self.compute = torch.cuda.Stream(), torch.cuda.Stream()
        self.copied = [torch.cuda.Event() for _ in self.sets]
        self.done = [torch.cuda.Event() for _ in self.sets]
        self.out = [torch.empty((2, max(packed.total_plans, 1)), dtype=torch.int64).pin_memory()
                    for _ in self.sets]
        self.k = 0

    def submit(self):
        """Enqueue one step; returns (ticket, bytes host->device, bytes device->host)."""
        slot = self.k % len(self.sets)
        self.k += 1
        d = self.sets[slot]
        self.copy.wait_event(self.done[slot])      # the set's previous step is finished
        d.load(self.copy)
        self.copied[slot].record(self.copy)
        self.compute.wait_event(self.copied[slot])
        import torch
        with torch.cuda.stream(self.compute):
            d.batch.eval(self.mask, self.compute, graph=True)
            n = self.packed.total_plans
            self.out[slot][0, :n].copy_(d.plan_s[:n], non_blocking=True)
            self.out[slot][1, :n].copy_(d.plan_rr[:n], non_blocking=True)
            self.done[slot].record(self.compute)
        return slot, self.packed.h2d_bytes, 2 * 8 * self.packed.total_plans

    def wait(self, ticket):
        self.done[ticket].synchronize()
        return self.out[ticket]

    def close(self):
        for d in self.sets:
            d.close()


# ----------------------------------------------------------------- surrogate

def wh_surrogate_features(layout, orders: wh_orders, plans: wh_plans, X, stream=None) -> None:
    _check(load().wh_surrogate_features(layout, ctypes.byref(orders), ctypes.byref(plans), ctypes.c_void_p(X),
                                        _stream_ptr(stream)), "wh_surrogate_features")


def wh_surrogate_create(seed: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().wh_surrogate_create(seed, ctypes.byref(h)), "wh_surrogate_create")
    return h


def wh_surrogate_set_params(s, params) -> None:
    import numpy as np
    p = np.ascontiguousarray(np.asarray(params, np.float32))
    assert p.size == WH_MLP_NPARAM
    _check(load().wh_surrogate_set_params(s, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
           "wh_surrogate_set_params")


def wh_surrogate_get_params(s):
    """(params, grads) as float32 numpy arrays."""
    import numpy as np
    p = np.zeros(WH_MLP_NPARAM, np.float32)
    g = np.zeros(WH_MLP_NPARAM, np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    _check(load().wh_surrogate_get_params(s, p.ctypes.data_as(fp), g.ctypes.data_as(fp)), "wh_surrogate_get_params")
    return p, g


def wh_batch_grow(layout, orders: wh_orders, slot_map, slot_map_stride: int, n_maps: int, max_orders: int,
                  max_lines: int, tour_off, order_seq, n_tours, stream=None) -> None:
    _check(load().wh_batch_grow(layout, ctypes.byref(orders), ctypes.c_void_p(slot_map), slot_map_stride, n_maps,
                                max_orders, max_lines, ctypes.c_void_p(tour_off), ctypes.c_void_p(order_seq),
                                ctypes.c_void_p(n_tours), _stream_ptr(stream)), "wh_batch_grow")


def wh_kmeans_slotting(layout, orders: wh_orders, signs, freq_weight: int, k: int, init, u, iters: int, x_out,
                       init_out, centroids, assign, slot_map, stream=None) -> None:
    _check(load().wh_kmeans_slotting(layout, ctypes.byref(orders), ctypes.c_void_p(signs), freq_weight, k,
                                     ctypes.c_void_p(init), ctypes.c_void_p(u), iters, ctypes.c_void_p(x_out),
                                     ctypes.c_void_p(init_out), ctypes.c_void_p(centroids), ctypes.c_void_p(assign),
                                     ctypes.c_void_p(slot_map), _stream_ptr(stream)), "wh_kmeans_slotting")


def wh_routes(layout, orders: wh_orders, plans: wh_plans, tours, n: int, max_points: int, points, n_points, length,
              stream=None) -> None:
    _check(load().wh_routes(layout, ctypes.byref(orders), ctypes.byref(plans), ctypes.c_void_p(tours), n, max_points,
                            ctypes.c_void_p(points), ctypes.c_void_p(n_points), ctypes.c_void_p(length),
                            _stream_ptr(stream)), "wh_routes")


def wh_surrogate_get_status(s) -> int:
    v = ctypes.c_uint32(0)
    _check(load().wh_surrogate_get_status(s, ctypes.byref(v)), "wh_surrogate_get_status")
    return int(v.value)


def wh_surrogate_predict(s, X, n: int, y, stream=None) -> None:
    _check(load().wh_surrogate_predict(s, ctypes.c_void_p(X), n, ctypes.c_void_p(y), _stream_ptr(stream)),
           "wh_surrogate_predict")


def wh_surrogate_predict_timeout_test(s, X, n: int, y, skip_tile: int, wait_ns: int, stream=None) -> None:
    _check(load().wh_surrogate_predict_timeout_test(s, ctypes.c_void_p(X), n, ctypes.c_void_p(y), skip_tile,
                                                    wait_ns, _stream_ptr(stream)),
           "wh_surrogate_predict_timeout_test")


def wh_surrogate_train_step(s, X, target, n: int, lr: float, loss=0, stream=None) -> None:
    _check(load().wh_surrogate_train_step(s, ctypes.c_void_p(X), ctypes.c_void_p(target), n, lr,
                                          ctypes.c_void_p(loss or None), _stream_ptr(stream)),
           "wh_surrogate_train_step")


def wh_surrogate_get_trace(s, which: int, dst, n_rows: int, stream=None) -> None:
    _check(load().wh_surrogate_get_trace(s, which, ctypes.c_void_p(dst), n_rows, _stream_ptr(stream)),
           "wh_surrogate_get_trace")


def wh_surrogate_screen(layout, s, orders: wh_orders, plans: wh_plans, moves, moves_per_plan: int, keep: int,
                        max_orders: int, max_lines: int, kept, y_tour=None, tour_changed=None, stream=None) -> None:
    _check(load().wh_surrogate_screen(layout, s, ctypes.byref(orders), ctypes.byref(plans), ctypes.c_void_p(moves),
                                      moves_per_plan, keep, max_orders, max_lines, ctypes.c_void_p(y_tour),
                                      ctypes.c_void_p(tour_changed), ctypes.c_void_p(kept), _stream_ptr(stream)),
           "wh_surrogate_screen")


def wh_surrogate_screen_eval(layout, s, orders: wh_orders, plans: wh_plans, moves, moves_per_plan: int, keep: int,
                             max_orders: int, max_lines: int, y_tour_cache, tour_changed, tour_s, tour_rr, kept,
                             kept_delta, kept_status, stream=None) -> None:
    _check(load().wh_surrogate_screen_eval(layout, s, ctypes.byref(orders), ctypes.byref(plans),
                                           ctypes.c_void_p(moves), moves_per_plan, keep, max_orders, max_lines,
                                           ctypes.c_void_p(y_tour_cache), ctypes.c_void_p(tour_changed),
                                           ctypes.c_void_p(tour_s), ctypes.c_void_p(tour_rr), ctypes.c_void_p(kept),
                                           ctypes.c_void_p(kept_delta), ctypes.c_void_p(kept_status),
                                           _stream_ptr(stream)), "wh_surrogate_screen_eval")


def wh_surrogate_screen_trace(layout):
    """(n_tasks, tasks, counted, features) device pointers of the layout's last screen."""
    n = ctypes.c_int64()
    t, c, f = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().wh_surrogate_screen_trace(layout, ctypes.byref(n), ctypes.byref(t), ctypes.byref(c),
                                            ctypes.byref(f)), "wh_surrogate_screen_trace")
    return n.value, t.value, c.value, f.value


class _DeviceView:
    """A device buffer owned by the library seen as an array (CUDA array
    interface), only for copying it into a torch tensor (torch takes no
    read-only views, so it is not marked read-only)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def wh_surrogate_destroy(s) -> None:
    load().wh_surrogate_destroy(s)


def unpack_params(p):
    """Packed parameter vector -> dict of arrays (w1 [192,256], b1, w2 [256,256], b2, w3, b3)."""
    sizes = (("w1", (192, 256)), ("b1", (256,)), ("w2", (256, 256)), ("b2", (256,)), ("w3", (256,)), ("b3", (1,)))
    out, off = {}, 0
    for k, shape in sizes:
        n = 1
        for d in shape:
            n *= d
        out[k] = p[off:off + n].reshape(shape)
        off += n
    return out


def pack_params(d):
    import numpy as np
    return np.concatenate([np.asarray(d[k], np.float32).reshape(-1) for k in ("w1", "b1", "w2", "b2", "w3", "b3")])


class Surrogate:
    """Owning wrapper of a ``wh_surrogate``."""

    def __init__(self, seed: int = 0):
        self.handle = wh_surrogate_create(seed)

    def set_params(self, packed):
        wh_surrogate_set_params(self.handle, packed)

    def params(self):
        return wh_surrogate_get_params(self.handle)

    def predict(self, X, stream=None):
        import torch
        n = int(X.shape[0])
        y = torch.empty(max(n, 1), dtype=torch.float32, device=X.device)
        wh_surrogate_predict(self.handle, X.data_ptr(), n, y.data_ptr(), stream)
        return y[:n]

    def status(self) -> int:
        """Read and clear the WH_STATUS_* bits of the prediction kernels (synchronises)."""
        return wh_surrogate_get_status(self.handle)

    def train_step(self, X, target, lr: float, stream=None):
        """Returns the loss (device tensor) before the step."""
        import torch
        loss = torch.zeros(1, dtype=torch.float32, device=X.device)
        wh_surrogate_train_step(self.handle, X.data_ptr(), target.data_ptr(), int(X.shape[0]), lr,
                                loss.data_ptr(), stream)
        return loss

    def trace(self, n_rows: int, stream=None) -> dict:
        """The last training step's intermediates (first n_rows rows): z1, h1,
        z2, h2 [n_rows, 256], y, dy [n_rows], dz2, dz1 [n_rows, 256]."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        spec = (("z1", WH_TRACE_Z1, torch.float32, 256), ("h1", WH_TRACE_H1, torch.bfloat16, 256),
                ("z2", WH_TRACE_Z2, torch.float32, 256), ("h2", WH_TRACE_H2, torch.bfloat16, 256),
                ("y", WH_TRACE_Y, torch.float32, 0), ("dy", WH_TRACE_DY, torch.float32, 0),
                ("dz2", WH_TRACE_DZ2, torch.bfloat16, 256), ("dz1", WH_TRACE_DZ1, torch.bfloat16, 256))
        out = {}
        for name, which, dt, cols in spec:
            t = torch.empty((max(n_rows, 1), cols) if cols else (max(n_rows, 1),), dtype=dt, device=dev)
            wh_surrogate_get_trace(self.handle, which, t.data_ptr(), n_rows, stream)
            out[name] = t[:n_rows]
        return out

    def close(self):
        if self.handle is not None and self.handle.value:
            wh_surrogate_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def features(layout: "Layout", prob: DeviceProblem, stream=None):
    """bf16 [n_tours, 192] features of every tour of `prob`."""
    import torch
    X = torch.empty((max(prob.n_tours, 1), WH_FEATURES), dtype=torch.bfloat16, device=prob.order_off.device)
    wh_surrogate_features(layout.handle, prob.orders(), prob.plans(), X.data_ptr(), stream)
    return X[:prob.n_tours]
