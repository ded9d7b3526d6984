#!/usr/bin/env python
"""Benchmark: exact tour evaluations per second on one GB300 (or N, weak scaling).

One step = one persistent launch, replayed as a CUDA graph, that scores 1,024
independent warehouse instances of uneven size (aisles U[8,64], slots per side
U[20,200], orders U[100,5000] of 1..12 lines, as many SKUs as locations with
Zipf(1.1) popularity slotted ABC with 10% swapped) with 256 random candidate
plans each (tours of at most 20 orders / 60 lines): every tour under both
routing rules (S-shape and optimal) and every plan's int64 sums.  Inputs are
synthetic (seeded generator) and resident in HBM when timing starts (about
3 GB of plan arrays, far above the L2 cache).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun each rank scores its own
1,024 instances (no collective on the data path); the timing is the max over
ranks.  Extra fields measure the other rows: the mid-size single-instance
launch, the paper-scale population, move deltas, the surrogate prescreen and
the next rows.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact tour evals/s (RR DP, S-shape) and surrogate-screened vs plain, 1 GB300"
UNIT = "tours/s"
N_INST, PLANS_PER_INST = 1024, 256
INST_SEED = 3
WORKLOAD = ("batched: 1,024 independent warehouse instances of uneven size (aisles U[8,64], slots/side "
            "U[20,200], orders U[100,5000] of 1-12 lines, SKUs = locations, Zipf(1.1) ABC-slotted with 10% "
            "swapped) x 256 random plans each (tours <= 20 orders / 60 lines), one persistent launch replayed "
            "as a CUDA graph; S-shape + optimal (Ratliff-Rosenthal) cost of every tour, int64 sum per plan")
PLANS_PER_STEP = 4096          # the mid-size launch (extra field "midsize")
MIDSIZE_WORKLOAD = ("midsize warehouse: 40 aisles x 100 slots/side (8,000 locations), 8,000 SKUs Zipf(1.1) "
                    "ABC-slotted with 10% swapped, 4,000 orders of 1-12 lines, 4,096 plans per step in tours "
                    "of <= 20 orders / 60 lines; S-shape + optimal (Ratliff-Rosenthal) cost of every tour, "
                    "int64 sum per plan")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batches", type=int, default=4, help="mid-size plan batches rotated across steps")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--midsize-steps", type=int, default=1000)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and move-delta measurements")
    ap.add_argument("--extra-steps", type=int, default=20)
    ap.add_argument("--ab-steps", type=int, default=100, help="plain local-search steps of the prescreen A/B")
    ap.add_argument("--train-steps", type=int, default=2500)
    ap.add_argument("--case", choices=["batched-small", "moves-small", "surrogate-small", "sshape-small", "train-small",
                                       "midsize-both"],
                    default=None,
                    help="run a small case of one kernel three times (for profiler captures) and exit")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.dev)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.seek(0)
        sm, mx, reasons, n = [], [], set(), 0
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            n += 1
            for name, v in zip(self.REASONS, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": n}


# ------------------------------------------------------------------ helpers

def algorithmic_bytes(inst):
    """Algorithmic HBM bytes of one evaluation, per unit and counted once
    (pick lists as if materialised, unpadded): 4 B per order line of every
    tour read, 4 B per tour offset, 4 B per tour per routing rule written
    (two rules), 8 B per plan per rule, and the slotting table (4 B per SKU)
    once per instance.  The kernel itself reads order ids (4 B per order, not
    per line), so its DRAM traffic is below this figure."""
    lines = int(inst.tour_lines().sum())
    return 4 * lines + 4 * (inst.n_tours + 1) + 8 * inst.n_tours + 16 * inst.n_plans + 4 * inst.n_sku


def algorithmic_bytes_one_rule(inst):
    """As algorithmic_bytes with one routing rule written (S-shape only)."""
    lines = int(inst.tour_lines().sum())
    return 4 * lines + 4 * (inst.n_tours + 1) + 4 * inst.n_tours + 8 * inst.n_plans + 4 * inst.n_sku


def dp_alg_ops(inst):
    """Algorithmic integer operations of the optimal-route DP over every tour
    of one evaluation (shared slotting): the Ratliff-Rosenthal programme in its
    standard form steps through every aisle from the depot's to the rightmost
    pick aisle r, 7 classes x 6 transitions + 7 x 5 per aisle, so
    sum over tours of (r + 1) * 77 (the kernel's reduced DP steps only over
    pick aisles; its sort, record scan and gather are not counted)."""
    import numpy as np
    L = inst.layout.slots_per_side
    line_aisle = (np.asarray(inst.slot_map, np.int64) // (2 * L))[np.asarray(inst.line_sku)]
    off = np.asarray(inst.order_off, np.int64)
    order_max = np.full(len(off) - 1, -1, np.int64)
    ne = np.diff(off) > 0
    order_max[ne] = np.maximum.reduceat(line_aisle, off[:-1][ne])
    to = np.asarray(inst.tour_off, np.int64)
    tour_max = np.full(len(to) - 1, -1, np.int64)
    nz = np.diff(to) > 0
    tour_max[nz] = np.maximum.reduceat(order_max[np.asarray(inst.order_seq)], to[:-1][nz])
    return int((tour_max + 1).sum()) * 77


def alu_peak_tops(dev, sm_max_mhz):
    """Integer issue limit of the GPU: one warp instruction per SM
    sub-partition per cycle, 4 sub-partitions x 32 lanes per SM, at the
    maximum SM clock (152 SMs x 128 x 2,070 MHz = 40.3 Tops/s on a GB300)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = sm_max_mhz or 2070.0
    return sms * 4 * 32 * mhz * 1e6 / 1e12


def run_sshape(wh, lay, probs, batches, costs, stream, steps):
    """The streaming path: the same plan batches scored under the S-shape
    rule alone (per-order aggregates built by k_prep on every call, then the
    sort-free streaming kernel).  Two rooflines: the streaming kernel alone
    (CUDA events around each launch) and the whole step (prep + kernel,
    back-to-back calls timed by two events, no per-kernel events)."""
    import torch
    for i in range(3):
        lay.eval_plans(probs[i % len(probs)], costs, 1, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    n_tours = 0
    for i in range(steps):
        lay.eval_plans(probs[i % len(probs)], costs, 1, stream)
        n_tours += batches[i % len(batches)].n_tours
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lay.set_timing(True)
    for i in range(steps):
        lay.eval_plans(probs[i % len(probs)], costs, 1, stream)
    kt = lay.timing()
    lay.set_timing(False)
    torch.cuda.synchronize()
    assert lay.status() == 0
    name, (launches, kms) = max(kt.items(), key=lambda kv: kv[1][1])
    per_launch_s = kms / 1e3 / max(launches, 1)
    alg = sum(algorithmic_bytes_one_rule(batches[i % len(batches)]) for i in range(steps)) / steps
    peak, kind = measured_peaks()
    achieved = alg / per_launch_s / 1e9
    step_s = ms / 1e3 / steps
    return {"workload": "the mid-size plan batches, S-shape rule only", "tours_per_s": n_tours / (ms / 1e3),
            "ms_per_step": ms / steps, "steps": steps,
            "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in kt.items()},
            "roofline": {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": kind, "algorithmic_bytes_per_launch": alg,
                         "launch_ms": per_launch_s * 1e3},
            "step_roofline": {"bound": "hbm", "achieved": alg / step_s / 1e9, "peak": peak, "unit": "GB/s",
                              "frac": alg / step_s / 1e9 / peak, "peak_kind": kind,
                              "note": "whole wh_eval_plans call: per-order aggregates (k_prep) + streaming kernel"}}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the plan-evaluation kernels' source (the committed ncu
    summaries name the source they were taken on)."""
    h = hashlib.sha256()
    for name in ("k_eval.cu", "tour_core.cuh"):
        with open(os.path.join(ROOT, "paper_2110_13693_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_profile():
    """The committed ncu summary of the dominant kernel (DRAM bytes per
    launch, issue and pipe utilisation), only if it was taken on the current
    kernel source."""
    path = os.path.join(ROOT, "profiles", "k_eval_short_midsize.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_sha") == kernel_source_hash():
            return d
    except Exception:
        pass
    return None


def make_batches(n_batches, rank):
    import wh_gen
    from paper_2110_13693_gb300.shard import plan_base
    return [wh_gen.midsize(seed=2, n_plans=PLANS_PER_STEP, plan_base=plan_base(rank, b, n_batches, PLANS_PER_STEP))
            for b in range(n_batches)]


def cpu_oracle_rate(inst, seconds, plans_per_chunk=8):
    """The oracle as it stands (single-threaded C), on consecutive plan
    chunks of `inst` until `seconds` of CPU work have run."""
    import oracle
    oracle.build()
    tours = 0
    plans = 0
    t0 = time.perf_counter()
    p = 0
    while True:
        sub = inst.subset_plans(range(p, min(p + plans_per_chunk, inst.n_plans)))
        oracle.eval_plans(sub)
        tours += sub.n_tours
        plans += sub.n_plans
        p = (p + plans_per_chunk) % inst.n_plans
        el = time.perf_counter() - t0
        if el >= seconds:
            return tours / el, tours, plans, el


_WORKER_INST = {}


def _oracle_chunks(job):
    """One host core (a spawned worker): the oracle on consecutive plan chunks
    of the mid-size workload, from plan `start`, for `seconds` of wall time;
    returns (tours, plans, seconds)."""
    seed, n_plans, start, seconds, per_chunk = job
    import oracle
    import wh_gen
    oracle.build()
    key = (seed, n_plans)
    if key not in _WORKER_INST:          # generated once per worker process
        _WORKER_INST[key] = wh_gen.midsize(seed=seed, n_plans=n_plans)
    inst = _WORKER_INST[key]
    tours = plans = 0
    p = start % n_plans
    t0 = time.perf_counter()
    while True:
        sub = inst.subset_plans(range(p, min(p + per_chunk, n_plans)))
        oracle.eval_plans(sub)
        tours += sub.n_tours
        plans += sub.n_plans
        p = (p + per_chunk) % n_plans
        el = time.perf_counter() - t0
        if el >= seconds:
            return tours, plans, el


def cpu_oracle_rate_all_cores(seconds, cores):
    """The same oracle on every host core: one spawned process per core, each
    on its own plan chunks (the plans are independent); tours per second of
    wall time."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    jobs = [(2, PLANS_PER_STEP, i * (PLANS_PER_STEP // cores), seconds, 8) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_chunks, jobs)
    tours = sum(r[0] for r in res)
    plans = sum(r[1] for r in res)
    el = max(r[2] for r in res)
    return tours / el, tours, plans, el


# ------------------------------------------------- other hot-path rows

def run_moves(wh, dev, steps, cpu=True):
    """Paper-scale local search: 500 aisles x 200 slots/side, 50,000 SKUs,
    16,384 plans with their own slottings, 64 moves per plan per step."""
    import numpy as np
    import torch
    import wh_gen
    n_plans, M = 16384, 64
    inst = wh_gen.paperscale(seed=4, n_plans=n_plans)
    lay = wh.Layout.of(inst.layout)
    base = wh.to_device(inst, dev)
    smap = base.slot_map.repeat(n_plans)
    prob = wh.DeviceProblem(base.order_off, base.line_sku, smap, base.plan_tour_off, base.tour_off,
                            base.order_seq, inst.n_sku, inst.n_sku)
    costs = wh.evaluate(lay, prob)
    moves = []
    for step in range(steps + 2):
        mv = wh_gen.gen_moves(17, step, inst, M)
        mv[..., 3] = np.arange(n_plans)[:, None]
        moves.append(torch.as_tensor(mv.reshape(-1, 4)).to(dev))
    for i in range(2):
        lay.eval_moves(prob, costs, moves[i], 24)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(steps):
        d, s = lay.eval_moves(prob, costs, moves[2 + i], 24)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    n_ok = int((s == 0).sum().item())
    walked, walked_lines = lay.move_stats()
    # algorithmic bytes of one call: per move its record (16 B), both deltas
    # (16 B) and its status (4 B); per changed tour walked its task record
    # (16 B), its two tour offsets and two current costs (16 B), and per line
    # of it the SKU and the SKU's location under the plan's slotting (8 B)
    mv_bytes = n_plans * M * 36 + walked * 32 + walked_lines * 8
    peak, kind = measured_peaks()
    mv_ach = mv_bytes / (el / steps) / 1e9
    o_mv = None
    if cpu:
        # the CPU baseline: the oracle on the first plan's 64 moves (each
        # re-scores the whole plan), single-threaded
        import oracle
        mv_c = moves[2][:M].cpu().numpy().copy()
        mv_c[:, 3] = 0
        tc = time.perf_counter()
        oracle.eval_moves(inst.subset_plans([0]), mv_c, 24, 0, slot_map=inst.slot_map, slot_map_stride=inst.n_sku)
        o_mv = time.perf_counter() - tc
    # full local-search steps (evaluate, apply, re-score) on the same population,
    # after one untimed step (first use of every kernel on the way)
    applied = lay.ls_step(prob, costs, moves[0], M, 24)
    int((applied >= 0).sum().item())
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    improved = 0
    for i in range(steps):
        applied = lay.ls_step(prob, costs, moves[2 + i], M, 24)
        improved += int((applied >= 0).sum().item())
    torch.cuda.synchronize()
    el2 = time.perf_counter() - t1
    # relocations into empty locations (150,000 of the 200,000 are empty in
    # every plan): occupancy bits built once, 64 relocations per plan
    lay.occupancy(prob)
    rel = []
    for step in range(steps + 1):
        mv = wh_gen.gen_relocations(18, step, inst, M)
        rel.append(torch.as_tensor(mv.reshape(-1, 4)).to(dev))
    lay.eval_moves(prob, costs, rel[0], 24)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    for i in range(steps):
        d, s = lay.eval_moves(prob, costs, rel[1 + i], 24)
    torch.cuda.synchronize()
    el3 = time.perf_counter() - t2
    n_rel_ok = int((s == 0).sum().item())
    assert lay.status() == 0
    lay.close()
    # the CPU baseline: the oracle on the 64 relocations of the first plan
    # (each re-scores the whole plan), single-threaded
    o_s = None
    if cpu:
        import oracle
        one_plan = inst.subset_plans([0])
        mv0 = rel[1][:M].cpu().numpy().copy()
        mv0[:, 3] = 0
        t0 = time.perf_counter()
        oracle.eval_moves(one_plan, mv0, 24, 0, slot_map=inst.slot_map, slot_map_stride=inst.n_sku)
        o_s = time.perf_counter() - t0
    return {"workload": "paper scale: 500 aisles x 200 slots/side, 50,000 SKUs Zipf(1.0), 4,000 orders, "
                        "16,384 plans x 64 moves per step (order swap / relocate / SKU-slot swap)",
            "moves_per_step": n_plans * M, "ms_per_step": el * 1e3 / steps,
            "move_deltas_per_s": n_plans * M * steps / el, "evaluated_fraction": n_ok / (n_plans * M),
            "changed_tours_per_step": walked, "changed_tour_lines_per_step": walked_lines,
            "roofline": {"bound": "hbm", "achieved": mv_ach, "peak": peak, "unit": "GB/s", "frac": mv_ach / peak,
                         "peak_kind": kind, "algorithmic_bytes_per_step": mv_bytes,
                         "note": "whole wh_eval_moves call (wall clock, one synchronisation per call)"},
            "ls_step_ms": el2 * 1e3 / steps, "plans_improved_per_step": improved / steps, "steps": steps,
            "cpu_baseline": None if o_mv is None else {
                "value": M / o_mv, "unit": "move deltas/s", "cores": 1, "kind": "oracle",
                "sample": f"the 64 moves of one plan, {o_mv:.3f} s"},
            "relocations": {"moves_per_step": n_plans * M, "ms_per_step": el3 * 1e3 / steps,
                            "move_deltas_per_s": n_plans * M * steps / el3,
                            "into_empty_fraction": n_rel_ok / (n_plans * M),
                            "cpu_baseline": None if o_s is None else {
                                "value": M / o_s, "unit": "move deltas/s", "cores": 1, "kind": "oracle",
                                "sample": f"the 64 relocations of one plan, {o_s:.3f} s"}},
            "timing": "wall clock around the calls (each call synchronises once)"}


def run_batch_grow(wh, dev, cpu=True):
    """Batch formation (seed and grow by exact optimal length) of the mid-size
    order book under 304 ABC slottings (each with its own 10 % of swaps), one
    CTA per slotting; quality: the formed plan's optimal cost against random
    plans of the same capacity under the same slotting."""
    import numpy as np
    import torch
    import wh_gen
    inst = wh_gen.midsize(seed=2, n_plans=64)
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst, dev)
    n_maps = 304
    maps = torch.as_tensor(np.stack([wh_gen.gen_slot_abc(100 + i, inst.layout, inst.n_sku, 0.1)
                                     for i in range(n_maps)]).astype(np.int32)).to(dev)
    lay.batch_grow(prob, maps[:1], 20, 60)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    tour_off, order_seq, n_tours = lay.batch_grow(prob, maps, 20, 60)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    assert lay.status() == 0 and int(n_tours.min().item()) > 0
    # the first slotting's formed plan against the generator's random plans
    nt = int(n_tours[0].item())
    m0 = maps[0].contiguous()
    formed = wh.DeviceProblem(prob.order_off, prob.line_sku, m0,
                              torch.tensor([0, nt], dtype=torch.int32, device=dev),
                              tour_off[0, :nt + 1].contiguous(), order_seq[0].contiguous(), inst.n_sku)
    rand = wh.DeviceProblem(prob.order_off, prob.line_sku, m0, prob.plan_tour_off, prob.tour_off, prob.order_seq,
                            inst.n_sku)
    f_cost = int(wh.evaluate(lay, formed).plan_rr[0].item())
    r_cost = wh.evaluate(lay, rand).plan_rr[:inst.n_plans].double().mean().item()
    # the CPU baseline on a bounded sample (the oracle's growth is quadratic
    # in the book): the first 400 orders under the first slotting, and the
    # kernel on the same 400 orders under all the slottings
    n_s = 400
    off_s = inst.order_off[:n_s + 1]
    lines_s = inst.line_sku[:off_s[-1]]
    sample = wh_gen.Instance(inst.layout, inst.n_sku, off_s, lines_s, inst.slot_map, inst.plan_tour_off,
                             inst.tour_off, inst.order_seq)
    o_s = None
    if cpu:
        import oracle
        t0 = time.perf_counter()
        oracle.batch_grow(inst.layout, off_s, lines_s, inst.n_sku, maps[0].cpu().numpy(), 20, 60)
        o_s = time.perf_counter() - t0
    sp = wh.to_device(sample, dev)
    lay.batch_grow(sp, maps[:1], 20, 60)
    torch.cuda.synchronize()
    e0.record()
    lay.batch_grow(sp, maps, 20, 60)
    e1.record()
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    lay.close()
    return {"workload": f"mid-size order book (4,000 orders) under {n_maps} ABC slottings, tours of <= 20 orders / "
                        "60 lines, one launch",
            "ms": ms, "orders_per_s": n_maps * inst.n_orders / (ms / 1e3),
            "tours_per_s": float(n_tours.double().sum().item()) / (ms / 1e3),
            "formed_plan_optimal_cost": f_cost, "random_plans_mean_optimal_cost": r_cost,
            "formed_over_random": f_cost / r_cost,
            "kernel_on_sample": {"sample": f"the first {n_s} orders under all {n_maps} slottings", "ms": ms_s,
                                 "orders_per_s": n_maps * n_s / (ms_s / 1e3)},
            "cpu_baseline": None if o_s is None else {
                "value": n_s / o_s, "unit": "orders/s", "cores": 1, "kind": "oracle",
                "sample": f"the first {n_s} orders under one slotting, {o_s:.2f} s"}}


def run_layout_sweep(wh, dev):
    """Layout sweep (Eq. (1) reading): the mid-size orders and 256 random
    plans on 4 aisle counts x 3 pitches of about 8,000 locations, each layout
    ABC-slotted and scored on the device; utilisation, feasibility (aisle width
    >= 1 picker width) and the Pareto front of utilisation against length."""
    import wh_gen
    from paper_2110_13693_gb300 import sweep
    inst = wh_gen.midsize(seed=2, n_plans=256)
    t0 = time.perf_counter()
    rows = sweep.layout_sweep(wh, inst, aisle_counts=[20, 40, 80, 100], pitches=[3, 4, 5], n_loc=8000,
                              rack_depth=1.0, k=1.0, delta=1.0, device=dev)
    el = time.perf_counter() - t0
    front = sweep.pareto(rows)
    return {"workload": "mid-size orders, 256 random plans, 12 layouts of ~8,000 locations "
                        "(aisles 20/40/80/100, pitch 3/4/5)",
            "layouts": len(rows), "seconds": el,
            "pareto": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()} for r in front]}


def run_kmeans(wh, dev, cpu=True):
    """K-means slotting on the category workloads: one call (features,
    K-means++ seeding, Lloyd rounds, zones) timed with CUDA events after a
    warm-up, and the slotting scored by the evaluator against the ABC one on
    the same random plans and on seed-and-grow plans formed under each."""
    import numpy as np
    import torch
    import wh_gen

    def one(inst, k, iters, fw):
        lay = wh.Layout.of(inst.layout)
        prob = wh.to_device(inst, dev)
        sg = torch.as_tensor(wh_gen.gen_signs(3, (inst.n_sku, 32))).to(dev)
        u = torch.as_tensor(np.array([wh_gen.stream_word(5, 11, i) for i in range(k)], np.uint64).view(np.int64)).to(dev)
        lay.kmeans_slotting(prob, sg, k, iters, fw, u=u)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x, seeds, cent, assign, smap = lay.kmeans_slotting(prob, sg, k, iters, fw, u=u)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        assert lay.status() == 0
        km = wh.DeviceProblem(prob.order_off, prob.line_sku, smap, prob.plan_tour_off, prob.tour_off,
                              prob.order_seq, inst.n_sku)
        abc_rand = wh.evaluate(lay, prob).plan_rr[:inst.n_plans].double().mean().item()
        km_rand = wh.evaluate(lay, km).plan_rr[:inst.n_plans].double().mean().item()
        row = {"ms": ms, "k": k, "iters": iters, "freq_weight": fw,
               "random_plans_optimal_abc": abc_rand, "random_plans_optimal_kmeans": km_rand,
               "kmeans_over_abc_random_plans": km_rand / abc_rand}
        if inst.layout.n_aisles <= 255:
            maps = torch.stack([prob.slot_map, smap])
            to, seq, nt = lay.batch_grow(prob, maps, 20, 60)
            costs = []
            for i in range(2):
                n_t = int(nt[i].item())
                formed = wh.DeviceProblem(prob.order_off, prob.line_sku, maps[i].contiguous(),
                                          torch.tensor([0, n_t], dtype=torch.int32, device=dev),
                                          to[i, :n_t + 1].contiguous(), seq[i].contiguous(), inst.n_sku)
                costs.append(int(wh.evaluate(lay, formed).plan_rr[0].item()))
            row.update({"grown_plan_optimal_abc": costs[0], "grown_plan_optimal_kmeans": costs[1],
                        "kmeans_over_abc_grown_plans": costs[1] / costs[0]})
        lay.close()
        return row

    mid = one(wh_gen.midsize_cat(seed=6, n_plans=256), 64, 20, 64)
    paper = one(wh_gen.paperscale_cat(seed=7, n_plans=256), 256, 20, 64)
    # the CPU baseline: the oracle on the same mid-size call
    if cpu:
        import oracle
        ic = wh_gen.midsize_cat(seed=6, n_plans=1)
        sg = wh_gen.gen_signs(3, (ic.n_sku, 32))
        uu = np.array([wh_gen.stream_word(5, 11, i) for i in range(64)], np.uint64)
        t0 = time.perf_counter()
        oracle.kmeans_slotting(ic.layout, ic.order_off, ic.line_sku, ic.n_sku, sg, 64, 64, 20, u=uu)
        o_ms = (time.perf_counter() - t0) * 1e3
        mid["cpu_baseline"] = {"value": o_ms, "unit": "ms per call", "cores": 1, "kind": "oracle",
                               "sample": "the same mid-size call (k = 64, 20 rounds)"}
    return {"workload": "category order books: mid-size (8,000 SKUs, 64 categories, 40 x 100 layout, k = 64) and "
                        "paper-scale (50,000 SKUs, 256 categories, 500 x 200 layout, k = 256), 20 Lloyd rounds",
            "midsize": mid, "paperscale": paper}


def run_routes(wh, dev, cpu=True):
    """Explicit optimal pick sequences for every tour of 1,024 paper-scale
    plans (one thread per tour: tracking DP, backtrack, Euler circuit), one
    launch after a warm-up; the route lengths are checked against the
    evaluator's optimal tour lengths."""
    import torch
    import wh_gen
    inst = wh_gen.paperscale(seed=4, n_plans=1024)
    lay = wh.Layout.of(inst.layout)
    prob = wh.to_device(inst, dev)
    tours = torch.arange(inst.n_tours, dtype=torch.int32, device=dev)
    lay.routes(prob, tours[:1024])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    pts, npt, length = lay.routes(prob, tours)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    assert lay.status() == 0
    rr = wh.evaluate(lay, prob).tour_rr[:inst.n_tours]
    assert torch.equal(length, rr)
    lay.close()
    # the CPU baseline: the oracle's optimal length (the DP alone, no
    # sequence) of the first 5,000 tours, single-threaded
    n_o, o_s = 5000, None
    if cpu:
        import oracle
        locs = []
        for t in range(n_o):
            ls = []
            for o in inst.order_seq[inst.tour_off[t]:inst.tour_off[t + 1]]:
                ls.extend(inst.slot_map[inst.line_sku[inst.order_off[o]:inst.order_off[o + 1]]].tolist())
            locs.append(ls)
        t0 = time.perf_counter()
        for ls in locs:
            oracle.rr(inst.layout, ls)
        o_s = time.perf_counter() - t0
    return {"workload": f"all {inst.n_tours:,} tours of 1,024 paper-scale plans, one launch",
            "ms": ms, "tours_per_s": inst.n_tours / (ms / 1e3),
            "points_per_s": float(npt.double().sum().item()) / (ms / 1e3), "lengths_equal_optimal": True,
            "cpu_baseline": None if o_s is None else {
                "value": n_o / o_s, "unit": "tours/s", "cores": 1, "kind": "oracle",
                "sample": f"optimal length (the DP alone, no sequence) of the first {n_o} tours, {o_s:.2f} s"}}


def run_surrogate_ab(wh, dev, steps, train_steps, cpu=True):
    """Config 5: the MLP prescreen on the paper-scale population.  Trained on
    ~10M exactly scored tours of the paper-scale generator (four random
    populations), judged on a held-out one, then plain exact search and
    screened search (64 moves per plan, 5 % kept) run from the same start."""
    import numpy as np
    import torch
    import wh_gen
    from paper_2110_13693_gb300 import search
    n_plans, M = 16384, 64
    inst0 = wh_gen.paperscale(seed=4, n_plans=n_plans)
    lay = wh.Layout.of(inst0.layout)
    t0 = time.perf_counter()
    Xs, ts = [], []
    for k in range(5):
        inst = inst0 if k == 0 else wh_gen.paperscale(seed=4, n_plans=n_plans, plan_base=k * n_plans)
        prob = wh.to_device(inst, dev)
        costs = wh.evaluate(lay, prob)
        X, t = search.training_set(wh, lay, prob, costs, inst.layout)
        Xs.append(X)
        ts.append(t)
    X_train, t_train = torch.cat(Xs[1:]), torch.cat(ts[1:])
    X_held, t_held = Xs[0][:500000], ts[0][:500000]
    data_s = time.perf_counter() - t0
    sg = wh.Surrogate(11)
    t1 = time.perf_counter()
    search.train(sg, X_train, t_train, train_steps, 4096, 2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    mean_err, p99_err = search.errors(sg, X_held, t_held)
    # inference on its own: the 500,000 held-out rows in one prediction
    sg.predict(X_held[:4096])
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    sg.predict(X_held)
    e1.record()
    torch.cuda.synchronize()
    infer = {"rows": int(X_held.shape[0]), "ms": e0.elapsed_time(e1),
             "rows_per_s": X_held.shape[0] / (e0.elapsed_time(e1) / 1e3)}
    if cpu:
        # the CPU baseline: the oracle's features and MLP forward (float64,
        # the same bf16 rounding points) of the first 2,000 tours, one core
        import oracle
        n_c = 2000
        w = {k: (oracle.bf16(v) if k in ("w1", "w2") else v) for k, v in wh.unpack_params(sg.params()[0]).items()}
        locs = []
        for t_i in range(n_c):
            ls = []
            for o in inst0.order_seq[inst0.tour_off[t_i]:inst0.tour_off[t_i + 1]]:
                ls.extend(inst0.slot_map[inst0.line_sku[inst0.order_off[o]:inst0.order_off[o + 1]]].tolist())
            locs.append(ls)
        tc = time.perf_counter()
        Xc = np.stack([oracle.bf16(oracle.features(inst0.layout, ls)) for ls in locs])
        oracle.mlp_forward(w, Xc)
        o_s = time.perf_counter() - tc
        infer["cpu_baseline"] = {"value": n_c / o_s, "unit": "tours/s (features + MLP forward)", "cores": 1,
                                 "kind": "oracle", "sample": f"the first {n_c} tours, {o_s:.2f} s"}
    del Xs, ts, X_train, t_train

    def moves_fn0(step):
        mv = wh_gen.gen_moves(22, step, inst0, M)
        mv[..., 3] = np.arange(n_plans)[:, None]
        return torch.as_tensor(mv.reshape(-1, 4)).to(dev)

    def population():
        base = wh.to_device(inst0, dev)
        smap = base.slot_map.repeat(n_plans)
        prob = wh.DeviceProblem(base.order_off, base.line_sku, smap, base.plan_tour_off, base.tour_off.clone(),
                                base.order_seq.clone(), inst0.n_sku, inst0.n_sku)
        return prob, wh.evaluate(lay, prob)

    keep = search.keep_count(M)

    def ab(seed):
        """Plain exact search (`steps` steps) and, from the same start over the
        same sequence of move sets, screened search with the trained network
        and screened search keeping a seeded random `keep` of the moves (the
        same exact re-scores without the network), both for twice as many
        steps; wall clock of every step."""
        moves = {}

        def moves_fn(step):
            if step not in moves:
                mv = wh_gen.gen_moves(seed, step, inst0, M)
                mv[..., 3] = np.arange(n_plans)[:, None]
                moves[step] = torch.as_tensor(mv.reshape(-1, 4)).to(dev)
            return moves[step]

        for st in range(steps * 2):
            moves_fn(st)                  # generated outside the timed searches
        gen = torch.Generator(device=dev).manual_seed(seed)
        rand_idx = {}

        def random_fn(step):
            if step not in rand_idx:
                rand_idx[step] = torch.argsort(torch.rand((n_plans, M), device=dev, generator=gen), dim=1)[:, :keep]
            mv = moves_fn(step).view(n_plans, M, 4)
            return mv[torch.arange(n_plans, device=dev)[:, None], rand_idx[step]].reshape(-1, 4).contiguous()

        for st in range(steps * 2):
            random_fn(st)
        prob, costs = population()
        start_best = int(costs.plan_rr[:n_plans].min().item())
        plain = search.run_search(wh, lay, prob, costs, moves_fn, steps, M, 24, 0)
        target = plain[-1][1]
        prob, costs = population()
        screened = search.run_search(wh, lay, prob, costs, moves_fn, steps * 2, M, 24, 0, sg=sg, keep=keep)
        prob, costs = population()
        rand = search.run_search(wh, lay, prob, costs, random_fn, steps * 2, keep, 24, 0)
        hit = next((tr[0] for tr in screened if tr[1] <= target), None)
        t_eq = plain[-1][0]
        best_at_eq = min((tr[1] for tr in screened if tr[0] <= t_eq), default=start_best)
        rand_at_eq = min((tr[1] for tr in rand if tr[0] <= t_eq), default=start_best)
        return {"move_seed": seed, "start_best": start_best,
                "plain": {"steps": len(plain), "seconds": plain[-1][0], "best": plain[-1][1], "mean": plain[-1][2],
                          "ms_per_step": plain[-1][0] * 1e3 / len(plain)},
                "screened": {"steps": len(screened), "seconds": screened[-1][0], "best": screened[-1][1],
                             "mean": screened[-1][2], "ms_per_step": screened[-1][0] * 1e3 / len(screened),
                             "seconds_to_plain_best": hit, "best_at_plain_wall_time": best_at_eq,
                             "mean_after_plain_steps": screened[steps - 1][2]},
                "random_keep": {"steps": len(rand), "seconds": rand[-1][0], "best": rand[-1][1], "mean": rand[-1][2],
                                "ms_per_step": rand[-1][0] * 1e3 / len(rand), "best_at_plain_wall_time": rand_at_eq,
                                "mean_after_plain_steps": rand[steps - 1][2]},
                "screened_reaches_plain_best_faster": hit is not None and hit < plain[-1][0]}

    # untrained warm-up of every arm on a throwaway population: the first use
    # of every kernel (ours and torch's) stays out of the timed searches
    prob, costs = population()
    search.run_search(wh, lay, prob, costs, lambda st: moves_fn0(st), 2, M, 24, 0)
    search.run_search(wh, lay, prob, costs, lambda st: moves_fn0(st), 2, M, 24, 0, sg=sg, keep=keep)
    runs = [ab(seed) for seed in (23, 24, 25)]
    assert lay.status() == 0
    sg.close()
    lay.close()
    first = runs[0]
    return {"workload": "paper scale, 16,384 plans with their own slottings, 64 moves per plan per step; "
                        f"surrogate trained on {4 * inst0.n_tours} exactly scored tours of the same generator",
            "surrogate_mean_rel_error": mean_err, "surrogate_p99_rel_error": p99_err, "inference": infer,
            "held_out_tours": 500000, "train_steps": train_steps, "batch": 4096, "train_seconds": train_s,
            "data_seconds": data_s, "keep_per_plan": keep, "start_best": first["start_best"],
            "plain": first["plain"], "screened": first["screened"], "random_keep": first["random_keep"],
            "screened_reaches_plain_best_faster": first["screened_reaches_plain_best_faster"],
            "seeds": runs,
            "screened_faster_all_seeds": all(r["screened_reaches_plain_best_faster"] for r in runs),
            "screened_beats_random_keep_all_seeds": all(
                r["screened"]["mean_after_plain_steps"] < r["random_keep"]["mean_after_plain_steps"] for r in runs)}


# ----------------------------------------------- batched workload helpers

def make_instances(rank):
    """This rank's 1,024 instances (rank r takes generator indices
    r*1024 .. r*1024+1023, so ranks score different instances)."""
    import wh_gen
    return [wh_gen.batched_instance(INST_SEED, rank * N_INST + i, n_plans=PLANS_PER_INST) for i in range(N_INST)]


_WORKER_BATCHED = {}


def _oracle_batched(job):
    """One host core (a spawned worker): the oracle on plan chunks of the
    batched instances `ids` (taken in turn, `per_chunk` plans at a time) for
    `seconds` of wall time, or exactly one chunk of each id when seconds is
    0; returns (tours, plans, seconds)."""
    ids, seconds, per_chunk = job
    import oracle
    import wh_gen
    oracle.build()
    tours = plans = 0
    t0 = time.perf_counter()
    k = 0
    while True:
        i = ids[k % len(ids)]
        if i not in _WORKER_BATCHED:
            _WORKER_BATCHED.clear()          # one instance held at a time
            _WORKER_BATCHED[i] = wh_gen.batched_instance(INST_SEED, i, n_plans=PLANS_PER_INST)
        inst = _WORKER_BATCHED[i]
        p0 = (k // len(ids)) * per_chunk % inst.n_plans
        sub = inst.subset_plans(range(p0, min(p0 + per_chunk, inst.n_plans)))
        oracle.eval_plans(sub)
        tours += sub.n_tours
        plans += sub.n_plans
        k += 1
        el = time.perf_counter() - t0
        if (seconds <= 0 and k >= len(ids)) or (seconds > 0 and el >= seconds):
            return tours, plans, el


def cpu_oracle_batched(seconds, cores, per_chunk=4):
    """The oracle on every host core over the batched workload: one spawned
    process per core, core c scoring plan chunks of instances c, c + cores,
    ... for `seconds`; tours per second of wall time."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    jobs = [(list(range(c, N_INST, cores))[:8], seconds, per_chunk) for c in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_batched, jobs)
    tours = sum(r[0] for r in res)
    plans = sum(r[1] for r in res)
    el = max(r[2] for r in res)
    return tours / el, tours, plans, el


def batched_profile(tours_per_launch):
    """The committed ncu summary of k_eval_batch (DRAM bytes of one launch
    on a smaller batch of the same generator), scaled to a full launch by
    the tours processed, only if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "k_eval_batch_batched.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_sha") == kernel_source_hash():
            scale = tours_per_launch / float(d["tours_per_launch"])
            return d, float(d["dram_bytes_per_launch"]) * scale
    except Exception:
        pass
    return None, None


# -------------------------------------------------------------- our arm

def run_midsize(wh, dev, rank, args):
    """The mid-size single-instance launch (4,096 plans per wh_eval_plans
    call, 4 rotated batches): kernel roofline, the S-shape streaming path,
    end to end from host memory, and the oracle on all host cores."""
    import numpy as np
    import torch
    batches = make_batches(args.batches, rank)
    lay = wh.Layout.of(batches[0].layout)
    probs = [wh.to_device(b, dev) for b in batches]
    tours = [p.n_tours for p in probs]
    costs = wh.alloc_costs(max(tours), PLANS_PER_STEP, dev)
    stream = torch.cuda.current_stream(dev)
    mask = wh.WH_ROUTE_SSHAPE | wh.WH_ROUTE_OPTIMAL
    steps = args.midsize_steps
    for i in range(max(3, args.warmup)):
        lay.eval_plans(probs[i % len(probs)], costs, mask, stream)
    torch.cuda.synchronize()
    assert lay.status() == 0, "device status flagged an input error"
    lay.set_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    n_tours = 0
    for i in range(steps):
        b = i % len(probs)
        lay.eval_plans(probs[b], costs, mask, stream)
        n_tours += tours[b]
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    ktime = lay.timing()
    lay.set_timing(False)
    assert lay.status() == 0
    dom_name, (dom_launches, dom_ms) = max(ktime.items(), key=lambda kv: kv[1][1])
    per_launch_s = dom_ms / 1e3 / max(dom_launches, 1)
    alg = sum(algorithmic_bytes(batches[i % len(batches)]) for i in range(steps)) / steps
    ops = sum(dp_alg_ops(batches[i % len(batches)]) for i in range(len(batches))) / len(batches)
    peak, peak_kind = measured_peaks()
    achieved = alg / per_launch_s / 1e9
    alu_peak = alu_peak_tops(dev, None)
    prof = recorded_profile()
    out = {"workload": MIDSIZE_WORKLOAD, "steps": steps, "ms_per_step": ms / steps,
           "tours_per_s": n_tours / (ms / 1e3), "plans_per_s": PLANS_PER_STEP * steps / (ms / 1e3),
           "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in ktime.items()},
           "roofline": {"bound": "alu", "kernel": dom_name, "achieved": ops / per_launch_s / 1e12, "peak": alu_peak,
                        "unit": "Tops/s", "frac": ops / per_launch_s / 1e12 / alu_peak,
                        "peak_kind": "derived: SMs x 4 sub-partitions x 32 lanes x 2,070 MHz (issue limit)",
                        "algorithmic_ops_per_launch": ops, "launch_ms": per_launch_s * 1e3,
                        "traffic": float(prof["dram_bytes_per_launch"]) if prof else None,
                        "issue_active_frac": prof.get("issue_active_frac") if prof else None,
                        "alu_pipe_frac": prof.get("alu_pipe_frac") if prof else None,
                        "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg}}}
    out["sshape_only"] = run_sshape(wh, lay, probs, batches, costs, stream, min(steps, 200))
    # end to end from pinned host memory: 16-bit order ids widened on the device
    host = []
    for b in batches:
        seq = b.order_seq.astype(np.uint16).view(np.int16)
        host.append(wh.DeviceProblem(*(torch.as_tensor(getattr(b, f)).pin_memory() for f in
                                       ("order_off", "line_sku", "slot_map", "plan_tour_off", "tour_off")),
                                     torch.as_tensor(seq).pin_memory(), b.n_sku))
    plan_outs = [torch.empty((2, PLANS_PER_STEP), dtype=torch.int64).pin_memory() for _ in probs]
    pipe = wh.HostPipeline(lay, [(p, costs) for p in probs], mask)
    for i in range(len(probs)):
        pipe.wait(pipe.submit(host[i], plan_outs[i])[0])
    torch.cuda.synchronize()
    e_steps = 40
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(pipe.copy)
    e_tours, h2d, d2h, prev = 0, 0, 0, None
    for i in range(e_steps):
        b = i % len(probs)
        ticket, h2d, d2h = pipe.submit(host[b], plan_outs[b])
        if prev is not None:
            pipe.wait(prev)
        prev = ticket
        e_tours += tours[b]
    e1.record(pipe.compute)
    pipe.wait(prev)
    torch.cuda.synchronize()
    out["e2e"] = {"value": e_tours / (e0.elapsed_time(e1) / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                  "d2h_bytes_per_step": d2h, "steps": e_steps}
    if not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        rate, ct, cp, el = cpu_oracle_rate_all_cores(args.cpu_seconds / 2, cores)
        out["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{cp} plans ({ct} tours) of the mid-size workload, {el:.1f} s on "
                                         f"{cores} host cores (one process per core)"}
    lay.close()
    return out


def run_paperscale_eval(wh, dev, steps):
    """Config 4's whole population scored in one call: 16,384 paper-scale
    plans (500 aisles x 200 slots/side, 50,000 SKUs, tours of <= 24 orders,
    30 % of them longer than 64 lines), each plan with its own slotting
    (16,384 slot maps), both rules."""
    import torch
    import wh_gen
    n_plans = 16384
    inst = wh_gen.paperscale(seed=4, n_plans=n_plans)
    lay = wh.Layout.of(inst.layout)
    base = wh.to_device(inst, dev)
    prob = wh.DeviceProblem(base.order_off, base.line_sku, base.slot_map.repeat(n_plans), base.plan_tour_off,
                            base.tour_off, base.order_seq, inst.n_sku, inst.n_sku)
    costs = wh.alloc_costs(prob.n_tours, n_plans, dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        lay.eval_plans(prob, costs, 3, stream)
    torch.cuda.synchronize()
    lay.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        lay.eval_plans(prob, costs, 3, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    kt = lay.timing()
    lay.set_timing(False)
    assert lay.status() == 0
    long_frac = float((inst.tour_lines() > 64).mean())
    lay.close()
    alg = algorithmic_bytes(inst) + 4 * inst.n_sku * (n_plans - 1)   # one slotting table per plan
    peak, kind = measured_peaks()
    return {"workload": "paper scale: 500 aisles x 200 slots/side, 50,000 SKUs Zipf(1.0), 4,000 orders, 16,384 "
                        "plans with their own slottings, tours <= 24 orders; both rules",
            "tours_per_step": inst.n_tours, "ms_per_step": ms, "tours_per_s": inst.n_tours / (ms / 1e3),
            "plans_per_s": n_plans / (ms / 1e3), "long_tour_fraction": long_frac, "steps": steps,
            "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in kt.items()},
            "step_roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                              "frac": alg / (ms / 1e3) / 1e9 / peak, "peak_kind": kind,
                              "algorithmic_bytes_per_step": alg}}


def bind_host_near_gpu(dev_index):
    """Restrict this process to the host CPUs local to the GPU (the PCI
    device's local_cpulist in sysfs), so that pinned host buffers allocated
    afterwards are placed, by first touch, in that CPU's memory: on a
    two-socket host the host-to-device copies then do not cross the link
    between the sockets.  Returns what was done, for the bench line."""
    import torch
    try:
        p = torch.cuda.get_device_properties(dev_index)
        bdf = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        base = f"/sys/bus/pci/devices/{bdf}"
        with open(f"{base}/local_cpulist") as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if not part:
                continue
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        cpus &= os.sched_getaffinity(0)
        node = None
        try:
            with open(f"{base}/numa_node") as f:
                node = int(f.read().strip())
        except (OSError, ValueError):
            pass
        if not cpus:
            return {"restricted": False, "why": f"no usable CPU in {spec!r}"}
        restricted = len(cpus) < len(os.sched_getaffinity(0))
        if restricted:
            os.sched_setaffinity(0, cpus)
        return {"restricted": restricted, "pci": bdf, "local_cpus": len(cpus), "gpu_numa_node": node}
    except Exception as e:   # no sysfs entry or older torch: leave the affinity alone
        return {"restricted": False, "why": str(e)[:80]}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2110_13693_gb300 as wh
    from paper_2110_13693_gb300 import build as whbuild

    rank, world, local = dist_env()
    assert world == args.gpus or world == 1, "--gpus must match the torchrun world size"
    torch.cuda.set_device(local)
    host_binding = bind_host_near_gpu(local)
    if world > 1:
        dist.init_process_group(backend="nccl", init_method="env://")
    if rank == 0 or world == 1:
        whbuild.build()
    if world > 1:
        dist.barrier()
    wh.load()
    dev = torch.device("cuda", local)
    mask = wh.WH_ROUTE_SSHAPE | wh.WH_ROUTE_OPTIMAL

    insts = make_instances(rank)
    packed = wh.PackedInstances(insts)
    alg = sum(algorithmic_bytes(i) for i in insts)
    ops = sum(dp_alg_ops(i) for i in insts)
    tours_step = packed.total_tours
    lines_step = sum(int(i.tour_lines().sum()) for i in insts)
    del insts
    dset = packed.device_set(dev)
    stream = torch.cuda.current_stream(dev)
    dset.load(stream)
    torch.cuda.synchronize()
    batch = dset.batch
    cache = os.path.join(ROOT, "paper_2110_13693_gb300", "autotune_cache.json")
    th, ch, hit = batch.autotune(mask, cache, stream)
    for _ in range(max(3, args.warmup)):
        batch.eval(mask, stream, graph=True)
    torch.cuda.synchronize()
    assert batch.status() == 0, "device status flagged an input error"

    # ---- timed region: exactly K graph replays
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.15)   # let the sampler's first line land
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        batch.eval(mask, stream, graph=True)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    assert batch.status() == 0

    # ---- the same steps launched eagerly with CUDA events around each kernel
    k_steps = min(args.steps, 50)
    batch.set_timing(True)
    for _ in range(k_steps):
        batch.eval(mask, stream)
    ktime = batch.timing()
    batch.set_timing(False)
    torch.cuda.synchronize()
    assert batch.status() == 0

    from paper_2110_13693_gb300.shard import combine
    elapsed_ms, total_tours = combine(elapsed_ms, tours_step * args.steps, dev)
    value = total_tours / (elapsed_ms / 1e3)

    # ---- end to end from pinned host memory through the same public API:
    # every step copies all instances' inputs in (order ids as 16-bit values,
    # which the batch kernel reads as they are) and every plan's costs back;
    # the copy of a step overlaps the evaluation of the previous one
    packed.pin()
    pipe = wh.PackedPipeline(packed, mask, tuning=batch.tuning())
    for _ in range(2):
        pipe.wait(pipe.submit()[0])
    torch.cuda.synchronize()
    e_steps = max(1, min(args.e2e_steps, args.steps))
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(pipe.copy)
    prev, h2d, d2h = None, 0, 0
    for _ in range(e_steps):
        ticket, h2d, d2h = pipe.submit()
        if prev is not None:
            pipe.wait(prev)            # the previous step's plan costs are on the host now
        prev = ticket
    e1.record(pipe.compute)
    pipe.wait(prev)
    torch.cuda.synchronize()
    e2e_ms, e_tours = combine(e0.elapsed_time(e1), tours_step * e_steps, dev)
    e2e_value = e_tours / (e2e_ms / 1e3)
    for d in pipe.sets:
        assert d.batch.status() == 0
    pipe.close()

    if rank != 0:
        dset.close()
        dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel
    dom_name, (dom_launches, dom_ms) = max(ktime.items(), key=lambda kv: kv[1][1])
    per_launch_s = dom_ms / 1e3 / max(dom_launches, 1)
    peak, peak_kind = measured_peaks()
    achieved = alg / per_launch_s / 1e9
    prof, traffic = batched_profile(tours_step)
    alu_peak = alu_peak_tops(dev, clk.get("sm_max_mhz"))
    launches_per_step = len(ktime)
    step_s = elapsed_ms / 1e3 / args.steps

    extra = {}
    if world == 1:
        extra["midsize"] = run_midsize(wh, dev, rank, args)
    if not args.no_extra and world == 1:
        extra["paperscale_eval"] = run_paperscale_eval(wh, dev, max(3, args.extra_steps // 2))
        extra["moves"] = run_moves(wh, dev, max(2, args.extra_steps // 4), cpu=not args.no_cpu_baseline)
        extra["surrogate"] = run_surrogate_ab(wh, dev, args.ab_steps, args.train_steps, cpu=not args.no_cpu_baseline)
        extra["batch_formation"] = run_batch_grow(wh, dev, cpu=not args.no_cpu_baseline)
        extra["layout_sweep"] = run_layout_sweep(wh, dev)
        extra["routes"] = run_routes(wh, dev, cpu=not args.no_cpu_baseline)
        extra["kmeans_slotting"] = run_kmeans(wh, dev, cpu=not args.no_cpu_baseline)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cores = os.cpu_count() or 1
        rate, ct, cp, el = cpu_oracle_batched(args.cpu_seconds, cores)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{cp} plans ({ct} tours) of the same 1,024 instances, {el:.1f} s on {cores} host cores "
                         "(one process per core, each on plan chunks of its own instances)"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "instances": N_INST, "plans_per_step": packed.total_plans,
                   "tours_per_step": tours_step, "lines_per_step": lines_step, "routing": "S-shape + optimal",
                   "launch": f"CUDA graph replay of one persistent launch (autotuned: {th} threads, "
                             f"{ch} chunks per work item{', from cache' if hit else ''})",
                   "l2": f"inputs larger than L2: {packed.h2d_bytes / 1e9:.2f} GB of packed instance arrays "
                         f"({2 * packed.seq16.numel() / 1e9:.2f} GB of them order ids, 16-bit values the kernel "
                         "reads directly) resident (> 129 MB L2)",
                   "parallelism": f"dp{world} (independent instances per GPU)",
                   "host_binding": host_binding},
        "plans_per_s": world * packed.total_plans * args.steps / (elapsed_ms / 1e3),
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e_steps},
        "gpu_launches": launches_per_step * args.steps,
        "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4),
                        "share": round(v[1] / max(sum(x[1] for x in ktime.values()), 1e-12), 4)}
                    for k, v in ktime.items()},
        "roofline": {"bound": "alu", "kernel": dom_name, "achieved": ops / per_launch_s / 1e12, "peak": alu_peak,
                     "unit": "Tops/s", "frac": ops / per_launch_s / 1e12 / alu_peak,
                     "peak_kind": "derived: SMs x 4 sub-partitions x 32 lanes x max SM clock (issue limit)",
                     "algorithmic_ops_per_launch": ops,
                     "ops_per_tour": ops / tours_step,
                     "launch_ms": per_launch_s * 1e3,
                     "launch_timing": f"CUDA events around each launch of {k_steps} eager steps "
                                      "(graph replays carry no per-kernel events)",
                     "step_frac": ops / step_s / 1e12 / alu_peak,
                     "traffic": traffic,
                     "issue_active_frac": prof.get("issue_active_frac") if prof else None,
                     "alu_pipe_frac": prof.get("alu_pipe_frac") if prof else None,
                     "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                             "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg,
                             "step_frac": alg / step_s / 1e9 / peak}},
        "cpu_baseline": cpu,
    }
    out.update(extra)
    print(json.dumps(out))
    dset.close()
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle as it stands on every host core, on the same workload and
    metric: each step, core c scores a bounded sample of plans of its own
    batched instances (the whole run is sized to end within minutes)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    per_plan_s = 0.004
    per_core = int(max(1, min(64, 120.0 / max(1, args.steps + args.warmup) / per_plan_s)))
    with mp.get_context("spawn").Pool(cores) as pool:
        def step(i):
            jobs = [([(i * cores + c) % N_INST], 0.0, per_core) for c in range(cores)]
            return sum(r[0] for r in pool.map(_oracle_batched, jobs))
        for i in range(args.warmup):
            step(i)
        t0 = time.perf_counter()
        n = 0
        for i in range(args.steps):
            n += step(args.warmup + i)
        el = time.perf_counter() - t0
    value = n / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "instances": N_INST, "plans_per_step": per_core * cores,
                      "note": "each step scores a bounded sample of the same workload with the CPU oracle: "
                              f"{per_core} plans of one instance on each of {cores} host cores"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{per_core} plans of one batched instance per core per step, "
                                      f"{cores} processes"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_case(name):
    """Small cases for profiler captures: 256 batched instances x 64 plans,
    paper-scale move deltas on 1,024 plans x 64 moves, or the surrogate's
    kernels (features, prescreen, tensor-core inference)."""
    import numpy as np
    import torch
    import paper_2110_13693_gb300 as wh
    import wh_gen
    from paper_2110_13693_gb300 import build as whbuild
    whbuild.build()
    wh.load()
    if name == "train-small":
        # three training steps of 4,096 paper-scale-like feature rows
        g = torch.Generator(device="cuda").manual_seed(0)
        X = torch.randint(0, 3, (4096, 192), device="cuda", generator=g).to(torch.bfloat16)
        t = torch.rand(4096, device="cuda", generator=g)
        sg = wh.Surrogate(1)
        for _ in range(3):
            sg.train_step(X, t, 1e-3)
        torch.cuda.synchronize()
        assert sg.status() == 0
        sg.close()
    elif name in ("sshape-small", "midsize-both"):
        # one mid-size batch (4,096 plans), three calls: the S-shape rule
        # alone, or both rules
        inst = wh_gen.midsize(seed=2, n_plans=PLANS_PER_STEP)
        lay = wh.Layout.of(inst.layout)
        prob = wh.to_device(inst)
        costs = wh.alloc_costs(prob.n_tours, prob.n_plans)
        for _ in range(3):
            lay.eval_plans(prob, costs, 1 if name == "sshape-small" else 3)
        torch.cuda.synchronize()
        assert lay.status() == 0
        lay.close()
    elif name == "batched-small":
        # 256 instances of the headline's generator x 64 plans through the
        # same packed device set (16-bit order ids read directly) and CTA
        # size as the headline; work items of 120 chunks (ten for each of the
        # CTA's 12 warps, as the headline's items split evenly) fill the GPU
        insts = [wh_gen.batched_instance(3, i, n_plans=64) for i in range(256)]
        d = wh.PackedInstances(insts).device_set()
        d.load()
        d.batch.set_tuning(384, 120, 1)
        for _ in range(3):
            d.batch.eval(3)
        torch.cuda.synchronize()
        assert d.batch.status() == 0
        d.close()
    elif name == "surrogate-small":
        # features of every tour of 1,024 paper-scale plans, one prescreen of
        # 64 moves per plan, and inference on 1M feature rows (384 MB, above L2)
        n = 1024
        inst = wh_gen.paperscale(seed=4, n_plans=n)
        lay = wh.Layout.of(inst.layout)
        base = wh.to_device(inst)
        prob = wh.DeviceProblem(base.order_off, base.line_sku, base.slot_map.repeat(n), base.plan_tour_off,
                                base.tour_off, base.order_seq, inst.n_sku, inst.n_sku)
        sg = wh.Surrogate(1)
        X = wh.features(lay, prob)
        mv = wh_gen.gen_moves(17, 0, inst, 64)
        mv[..., 3] = np.arange(n)[:, None]
        lay.screen(sg, prob, torch.as_tensor(mv.reshape(-1, 4)).cuda(), 64, 4, 24)
        g = torch.Generator(device="cuda").manual_seed(0)
        Xr = torch.randint(0, 3, (1 << 20, 192), device="cuda", generator=g).to(torch.bfloat16)
        for _ in range(3):
            sg.predict(Xr)
        torch.cuda.synchronize()
        assert lay.status() == 0 and sg.status() == 0 and X.shape[0] == prob.n_tours
        sg.close()
        lay.close()
    else:
        n = 1024
        inst = wh_gen.paperscale(seed=4, n_plans=n)
        lay = wh.Layout.of(inst.layout)
        base = wh.to_device(inst)
        prob = wh.DeviceProblem(base.order_off, base.line_sku, base.slot_map.repeat(n), base.plan_tour_off,
                                base.tour_off, base.order_seq, inst.n_sku, inst.n_sku)
        costs = wh.evaluate(lay, prob)
        for step in range(3):
            mv = wh_gen.gen_moves(17, step, inst, 64)
            mv[..., 3] = np.arange(n)[:, None]
            lay.eval_moves(prob, costs, torch.as_tensor(mv.reshape(-1, 4)).cuda(), 24)
        torch.cuda.synchronize()
        assert lay.status() == 0
        lay.close()
    print(json.dumps({"case": name, "ok": True}))


def main():
    args = parse()
    if args.case:
        run_case(args.case)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
