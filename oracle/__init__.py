"""CPU ORACLE -- test infrastructure, not part of the product path.

Python loader for the plain single-threaded C evaluator in ``wh_oracle.c``.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the CUDA library never does, and this
package imports nothing from it.

Functions and the independent checks that pin them (all in ``tests/``):

* ``dist``           -- grid distance; pinned by Dijkstra (scipy) on the
                        explicit aisle/cross-aisle graph, all pairs, several
                        layouts (the paper names Dijkstra, Sec. 5).
* ``sshape``         -- S-shape walk; pinned by the closed form
                        2*x_r + (m even ? m*Y : (m-1)*Y + 2*d_r) and by
                        hand-drawn tours.
* ``heldkarp`` / ``permutation`` -- exact optimum on small tours; pinned
                        against each other and against a pure-Python
                        enumeration over scipy shortest paths.
* ``rr``             -- Ratliff-Rosenthal DP; pinned by Held-Karp on
                        thousands of random tours of <= 10 picks and by the
                        route invariants (opt <= S-shape, lower bound, even,
                        monotone in the pick set, ...).
* ``eval_plans``     -- plan sums; pinned by summing per-tour calls over
                        hand-assembled pick lists.
* ``ls_step``        -- one best-improvement local-search step, editing the
                        plans in place; pinned by checking the applied index
                        against the argmin of ``eval_moves`` and the new plan
                        cost against old cost + delta.
* ``features``       -- the 192 surrogate features of a tour; pinned by a
                        brute-force Python computation from the pick set.
* ``mlp_forward`` / ``mlp_backward`` / ``adam`` -- the surrogate MLP;
                        forward pinned by torch's float64 Linear + exact GELU
                        with the same bf16 rounding points, backward by
                        finite differences and by torch autograd, Adam by
                        torch.optim.Adam.
* ``mlp_train_trace`` -- one training step with every intermediate and the
                        backward's bf16 rounding points; pinned by torch
                        autograd with the same roundings as gradient hooks.
* ``kmeans_features`` / ``kmeans_slotting`` -- K-means slotting; features
                        pinned by the dense co-occurrence matrix times the
                        sign matrix (numpy) and exact integer square roots;
                        the clustering by scikit-learn's Lloyd K-means on
                        separated blobs (same assignment), the fixed point
                        (every SKU at its nearest centroid, every centroid
                        the rounded mean of its members) and hand-sized
                        cases; the placement by its definition (a bijection
                        onto the first n_sku aisle-major locations, clusters
                        in weight order, SKUs in frequency order).
* ``eval_moves``     -- move deltas by applying each move to a copy and
                        re-scoring the plan; pinned by building the moved
                        plans explicitly in Python and differencing two
                        ``eval_plans`` results, and by status special cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, portable C99) into liboracle.so."""
    srcs = [os.path.join(_HERE, f) for f in ("wh_oracle.c", "wh_oracle.h")]
    newest = max(os.path.getmtime(s) for s in srcs)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp,
                               os.path.join(_HERE, "wh_oracle.c")])
        os.replace(tmp, _SO)
    return _SO


class OrLayout(ctypes.Structure):
    _fields_ = [("n_aisles", ctypes.c_int32), ("slots_per_side", ctypes.c_int32),
                ("aisle_pitch", ctypes.c_int32), ("slot_pitch", ctypes.c_int32),
                ("cross_aisle_width", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            lp = ctypes.POINTER(OrLayout)
            lib.or_dist.restype = ctypes.c_int64
            lib.or_dist.argtypes = [lp] + [ctypes.c_int32] * 4
            for name in ("or_sshape_tour", "or_rr_tour", "or_heldkarp_tour", "or_permutation_tour"):
                f = getattr(lib, name)
                f.restype = ctypes.c_int64
                f.argtypes = [lp, i32p, ctypes.c_int32]
            lib.or_eval_plans.restype = ctypes.c_int
            lib.or_eval_plans.argtypes = [lp, ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p, ctypes.c_int64,
                                          ctypes.c_int32, i32p, i32p, i32p, i32p, i32p, i64p, i64p]
            lib.or_eval_moves.restype = ctypes.c_int
            lib.or_eval_moves.argtypes = [lp, ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p, ctypes.c_int64,
                                          ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, i64p, i32p]
            lib.or_batch_grow.restype = ctypes.c_int
            lib.or_batch_grow.argtypes = [lp, ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p, ctypes.c_int32,
                                          ctypes.c_int32, i32p, i32p, i32p]
            lib.or_kmeans_features.restype = ctypes.c_int
            lib.or_kmeans_features.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_int32, i32p, i32p]
            lib.or_kmeans_slotting.restype = ctypes.c_int
            lib.or_kmeans_slotting.argtypes = [lp, ctypes.c_int32, i32p, i32p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_int32, i32p, i32p, i32p, i32p, i32p]
            lib.or_kmeans_lloyd.restype = ctypes.c_int
            lib.or_kmeans_lloyd.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, i32p, i32p]
            lib.or_kmeans_pp_init.restype = ctypes.c_int
            lib.or_kmeans_pp_init.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, i32p]
            lib.or_ls_step.restype = ctypes.c_int
            lib.or_ls_step.argtypes = [lp, ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p, ctypes.c_int64,
                                       ctypes.c_int32, i32p, i32p, i32p, i32p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, i32p]
            f32p = ctypes.POINTER(ctypes.c_float)
            f64p = ctypes.POINTER(ctypes.c_double)
            lib.or_features.restype = ctypes.c_int
            lib.or_features.argtypes = [lp, i32p, ctypes.c_int32, f32p]
            lib.or_bf16.restype = ctypes.c_float
            lib.or_bf16.argtypes = [ctypes.c_float]
            lib.or_mlp_forward.restype = None
            lib.or_mlp_forward.argtypes = [f32p] * 7 + [ctypes.c_int32, f64p]
            lib.or_mlp_backward.restype = ctypes.c_double
            lib.or_mlp_backward.argtypes = [f32p] * 7 + [f64p, ctypes.c_int32] + [f64p] * 6
            lib.or_mlp_train_trace.restype = ctypes.c_double
            lib.or_mlp_train_trace.argtypes = [f32p] * 7 + [f64p, ctypes.c_int32] + [f64p] * 17
            lib.or_adam.restype = None
            lib.or_adam.argtypes = [f64p, f64p, f64p, f64p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int32]
            _lib = lib
    return _lib


def _layout(lay) -> OrLayout:
    return OrLayout(lay.n_aisles, lay.slots_per_side, lay.aisle_pitch, lay.slot_pitch, lay.cross_aisle_width)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a, t=ctypes.c_int32):
    return a.ctypes.data_as(ctypes.POINTER(t))


def dist(lay, a1: int, y1: int, a2: int, y2: int) -> int:
    return int(_load().or_dist(ctypes.byref(_layout(lay)), a1, y1, a2, y2))


def _tour(fn, lay, locs) -> int:
    arr = _i32(locs)
    v = int(fn(ctypes.byref(_layout(lay)), _ptr(arr), arr.shape[0]))
    if v < 0:
        raise ValueError(f"oracle error {v}")
    return v


def sshape(lay, locs) -> int:
    return _tour(_load().or_sshape_tour, lay, locs)


def rr(lay, locs) -> int:
    return _tour(_load().or_rr_tour, lay, locs)


def heldkarp(lay, locs) -> int:
    return _tour(_load().or_heldkarp_tour, lay, locs)


def permutation(lay, locs) -> int:
    return _tour(_load().or_permutation_tour, lay, locs)


def eval_plans(inst, slot_map=None, slot_map_stride: int = 0):
    """Per-tour and per-plan S-shape and optimal costs of an Instance:
    (tour_s int32, tour_rr int32, plan_s int64, plan_rr int64)."""
    lib = _load()
    smap = _i32(inst.slot_map if slot_map is None else slot_map)
    off, lines = _i32(inst.order_off), _i32(inst.line_sku)
    pto, to, seq = _i32(inst.plan_tour_off), _i32(inst.tour_off), _i32(inst.order_seq)
    nt, npl = to.shape[0] - 1, pto.shape[0] - 1
    ts, tr = np.zeros(max(nt, 1), np.int32), np.zeros(max(nt, 1), np.int32)
    ps, pr = np.zeros(max(npl, 1), np.int64), np.zeros(max(npl, 1), np.int64)
    rc = lib.or_eval_plans(ctypes.byref(_layout(inst.layout)), off.shape[0] - 1, _ptr(off), _ptr(lines),
                           inst.n_sku, _ptr(smap), slot_map_stride, npl, _ptr(pto), _ptr(to), _ptr(seq),
                           _ptr(ts), _ptr(tr), _ptr(ps, ctypes.c_int64), _ptr(pr, ctypes.c_int64))
    if rc != 0:
        raise ValueError(f"or_eval_plans error {rc}")
    return ts[:nt], tr[:nt], ps[:npl], pr[:npl]


def eval_moves(inst, moves, max_orders: int = 0, max_lines: int = 0, slot_map=None, slot_map_stride: int = 0):
    """Deltas [n, 2] (S-shape, optimal) and status [n] of moves {type, a, b, plan}."""
    lib = _load()
    smap = _i32(inst.slot_map if slot_map is None else slot_map)
    off, lines = _i32(inst.order_off), _i32(inst.line_sku)
    pto, to, seq = _i32(inst.plan_tour_off), _i32(inst.tour_off), _i32(inst.order_seq)
    mv = _i32(np.asarray(moves).reshape(-1, 4))
    n = mv.shape[0]
    delta = np.zeros((max(n, 1), 2), np.int64)
    status = np.zeros(max(n, 1), np.int32)
    rc = lib.or_eval_moves(ctypes.byref(_layout(inst.layout)), off.shape[0] - 1, _ptr(off), _ptr(lines), inst.n_sku,
                           _ptr(smap), slot_map_stride, pto.shape[0] - 1, _ptr(pto), _ptr(to), _ptr(seq), _ptr(mv), n,
                           max_orders, max_lines, _ptr(delta, ctypes.c_int64), _ptr(status))
    if rc != 0:
        raise ValueError(f"or_eval_moves error {rc}")
    return delta[:n], status[:n]


def batch_grow(layout, order_off, line_sku, n_sku: int, slot_map, max_orders: int, max_lines: int):
    """Seed-and-grow batching of the orders into tours (see or_batch_grow):
    (tour_off [n_tours + 1], order_seq [n_orders]) of one plan."""
    lib = _load()
    off, lines, smap = _i32(order_off), _i32(line_sku), _i32(slot_map)
    n_orders = off.shape[0] - 1
    to = np.zeros(n_orders + 1, np.int32)
    seq = np.zeros(max(n_orders, 1), np.int32)
    nt = ctypes.c_int32(0)
    rc = lib.or_batch_grow(ctypes.byref(_layout(layout)), n_orders, _ptr(off), _ptr(lines), n_sku, _ptr(smap),
                           max_orders, max_lines, _ptr(to), _ptr(seq), ctypes.byref(nt))
    if rc != 0:
        raise ValueError(f"or_batch_grow error {rc}")
    return to[:nt.value + 1].copy(), seq[:n_orders].copy()


KM_DIM, KM_SKETCH, KM_SCALE = 32, 31, 1024


def kmeans_features(order_off, line_sku, n_sku: int, signs, freq_weight: int):
    """(x [n_sku, 32] int32, freq [n_sku] int32): steps 1-2 of or_kmeans_slotting."""
    lib = _load()
    off, lines = _i32(order_off), _i32(line_sku)
    sg = np.ascontiguousarray(signs, dtype=np.int8).reshape(n_sku, KM_DIM)
    x = np.zeros((n_sku, KM_DIM), np.int32)
    freq = np.zeros(n_sku, np.int32)
    rc = lib.or_kmeans_features(off.shape[0] - 1, _ptr(off), _ptr(lines), n_sku, sg.ctypes.data, freq_weight,
                                _ptr(x), _ptr(freq))
    if rc != 0:
        raise ValueError(f"or_kmeans_features error {rc}")
    return x, freq


def kmeans_lloyd(x, centroids, iters: int):
    """Lloyd rounds from the given centroids: (centroids [k, 32], assign [n])."""
    lib = _load()
    xx = np.ascontiguousarray(x, dtype=np.int32).reshape(-1, KM_DIM)
    cent = np.array(centroids, dtype=np.int32).reshape(-1, KM_DIM).copy()
    assign = np.zeros(xx.shape[0], np.int32)
    rc = lib.or_kmeans_lloyd(_ptr(xx), xx.shape[0], cent.shape[0], iters, _ptr(cent), _ptr(assign))
    if rc != 0:
        raise ValueError(f"or_kmeans_lloyd error {rc}")
    return cent, assign


def kmeans_pp_init(x, k: int, u):
    """K-means++ seeds (SKU ids) of the feature rows x from draws u (uint64 [k])."""
    lib = _load()
    xx = np.ascontiguousarray(x, dtype=np.int32).reshape(-1, KM_DIM)
    uu = np.ascontiguousarray(u, dtype=np.uint64)
    init = np.zeros(k, np.int32)
    rc = lib.or_kmeans_pp_init(_ptr(xx), xx.shape[0], k, uu.ctypes.data, _ptr(init))
    if rc != 0:
        raise ValueError(f"or_kmeans_pp_init error {rc}")
    return init


def kmeans_slotting(layout, order_off, line_sku, n_sku: int, signs, freq_weight: int, k: int, iters: int,
                    init=None, u=None):
    """K-means slotting (see or_kmeans_slotting), seeded by the SKU ids `init`
    or, when it is None, by K-means++ from the uint64 draws `u`: (x [n_sku,
    32], seeds [k], centroids [k, 32], assign [n_sku], slot_map [n_sku])."""
    lib = _load()
    off, lines = _i32(order_off), _i32(line_sku)
    ini = None if init is None else _i32(init)
    uu = None if u is None else np.ascontiguousarray(u, dtype=np.uint64)
    sg = np.ascontiguousarray(signs, dtype=np.int8).reshape(n_sku, KM_DIM)
    x = np.zeros((n_sku, KM_DIM), np.int32)
    seeds = np.zeros(k, np.int32)
    cent = np.zeros((k, KM_DIM), np.int32)
    assign = np.zeros(n_sku, np.int32)
    smap = np.zeros(n_sku, np.int32)
    rc = lib.or_kmeans_slotting(ctypes.byref(_layout(layout)), off.shape[0] - 1, _ptr(off), _ptr(lines), n_sku,
                                sg.ctypes.data, freq_weight, k, None if ini is None else ini.ctypes.data,
                                None if uu is None else uu.ctypes.data, iters, _ptr(x), _ptr(seeds), _ptr(cent),
                                _ptr(assign), _ptr(smap))
    if rc != 0:
        raise ValueError(f"or_kmeans_slotting error {rc}")
    return x, seeds, cent, assign, smap


def ls_step(inst, moves, moves_per_plan: int, max_orders: int = 0, max_lines: int = 0, slot_map=None,
            slot_map_stride: int = 0):
    """Apply one local-search step to copies of the plans: returns
    (tour_off, order_seq, slot_map, applied) after the step."""
    lib = _load()
    smap = _i32(inst.slot_map if slot_map is None else slot_map).copy()
    off, lines = _i32(inst.order_off), _i32(inst.line_sku)
    pto, to, seq = _i32(inst.plan_tour_off), _i32(inst.tour_off).copy(), _i32(inst.order_seq).copy()
    mv = _i32(np.asarray(moves).reshape(-1, 4))
    npl = pto.shape[0] - 1
    applied = np.zeros(max(npl, 1), np.int32)
    rc = lib.or_ls_step(ctypes.byref(_layout(inst.layout)), off.shape[0] - 1, _ptr(off), _ptr(lines), inst.n_sku,
                        _ptr(smap), slot_map_stride, npl, _ptr(pto), _ptr(to), _ptr(seq), _ptr(mv), moves_per_plan,
                        max_orders, max_lines, _ptr(applied))
    if rc != 0:
        raise ValueError(f"or_ls_step error {rc}")
    return to, seq, smap, applied[:npl]


MLP_IN, MLP_H = 192, 256


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def features(lay, locs) -> np.ndarray:
    """float32[192] features of one tour (before bf16 rounding)."""
    arr = _i32(locs)
    out = np.zeros(192, np.float32)
    rc = _load().or_features(ctypes.byref(_layout(lay)), _ptr(arr), arr.shape[0], _ptr(out, ctypes.c_float))
    if rc != 0:
        raise ValueError(f"or_features error {rc}")
    return out


def bf16(x) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest even), returned as float32."""
    f = _load().or_bf16
    a = np.asarray(x, np.float32)
    return np.vectorize(lambda v: f(float(v)), otypes=[np.float32])(a)


def mlp_forward(params, X) -> np.ndarray:
    """params: dict w1 [192,256], b1, w2 [256,256], b2, w3 [256], b3 [1] (bf16 values)."""
    X = _f32(X)
    n = X.shape[0]
    y = np.zeros(max(n, 1), np.float64)
    ps = [_f32(params[k]) for k in ("w1", "b1", "w2", "b2", "w3", "b3")]
    _load().or_mlp_forward(*[_ptr(p, ctypes.c_float) for p in ps], _ptr(X, ctypes.c_float), n,
                           _ptr(y, ctypes.c_double))
    return y[:n]


def mlp_backward(params, X, t):
    """(loss, grads dict) of 0.5 * mean((y - t)^2)."""
    X = _f32(X)
    t = np.ascontiguousarray(np.asarray(t, np.float64))
    n = X.shape[0]
    g = {"w1": np.zeros((MLP_IN, MLP_H)), "b1": np.zeros(MLP_H), "w2": np.zeros((MLP_H, MLP_H)),
         "b2": np.zeros(MLP_H), "w3": np.zeros(MLP_H), "b3": np.zeros(1)}
    ps = [_f32(params[k]) for k in ("w1", "b1", "w2", "b2", "w3", "b3")]
    loss = _load().or_mlp_backward(*[_ptr(p, ctypes.c_float) for p in ps], _ptr(X, ctypes.c_float),
                                   _ptr(t, ctypes.c_double), n,
                                   *[_ptr(g[k], ctypes.c_double) for k in ("w1", "b1", "w2", "b2", "w3", "b3")])
    return float(loss), g


TRACE_ROWS = ("z1", "h1", "z2", "h2", "d2pre", "d2", "s1", "d1pre", "d1")


def mlp_train_trace(params, X, t):
    """(loss, trace dict, grads dict) of one training step with the bf16
    rounding points of the tensor-core contract: activations h1, h2 and the
    back-propagated d2 = dL/dz2, d1 = dL/dz1 rounded to bf16 before use.
    trace: z1, h1, z2, h2, d2pre, d2, s1, d1pre, d1 [n, 256]; y, dy [n]."""
    X = _f32(X)
    t = np.ascontiguousarray(np.asarray(t, np.float64))
    n = X.shape[0]
    tr = {k: np.zeros((n, MLP_H)) for k in TRACE_ROWS}
    tr["y"], tr["dy"] = np.zeros(n), np.zeros(n)
    g = {"w1": np.zeros((MLP_IN, MLP_H)), "b1": np.zeros(MLP_H), "w2": np.zeros((MLP_H, MLP_H)),
         "b2": np.zeros(MLP_H), "w3": np.zeros(MLP_H), "b3": np.zeros(1)}
    ps = [_f32(params[k]) for k in ("w1", "b1", "w2", "b2", "w3", "b3")]
    order = ("z1", "h1", "z2", "h2", "y", "dy", "d2pre", "d2", "s1", "d1pre", "d1")
    loss = _load().or_mlp_train_trace(*[_ptr(p, ctypes.c_float) for p in ps], _ptr(X, ctypes.c_float),
                                      _ptr(t, ctypes.c_double), n,
                                      *[_ptr(tr[k], ctypes.c_double) for k in order],
                                      *[_ptr(g[k], ctypes.c_double) for k in ("w1", "b1", "w2", "b2", "w3", "b3")])
    return float(loss), tr, g


def adam(p, m, v, g, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = np.ascontiguousarray(g, np.float64)
    _load().or_adam(_ptr(p, ctypes.c_double), _ptr(m, ctypes.c_double), _ptr(v, ctypes.c_double),
                    _ptr(g, ctypes.c_double), p.size, lr, b1, b2, eps, step)
