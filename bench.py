#!/usr/bin/env python
"""Benchmark: exact tour evaluations per second on one GB300 (or N, weak scaling).

One step = one call of wh_eval_plans on a batch of 4,096 candidate plans of
the mid-size warehouse (40 aisles x 100 slots per side, 8,000 SKUs with
Zipf(1.1) popularity slotted ABC with 10% swapped, 4,000 orders of 1..12
lines, tours of at most 20 orders / 60 lines), scoring every tour under both
routing rules (S-shape and optimal) and every plan's int64 sums.  Inputs are
synthetic (seeded generator) and resident in HBM when timing starts; steps
rotate over several plan batches whose combined size exceeds the L2 cache.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun each rank scores its own
batches (no collective on the data path); the timing is the max over ranks.
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
PLANS_PER_STEP = 4096
WORKLOAD = ("midsize warehouse: 40 aisles x 100 slots/side (8,000 locations), 8,000 SKUs Zipf(1.1) "
            "ABC-slotted with 10% swapped, 4,000 orders of 1-12 lines, 4,096 plans per step in tours "
            "of <= 20 orders / 60 lines; S-shape + optimal (Ratliff-Rosenthal) cost of every tour, "
            "int64 sum per plan")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batches", type=int, default=4, help="plan batches rotated across steps")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
    """HBM bytes one evaluation must move at least, counted once: the plans'
    order sequences and tour offsets read, two int32 costs per tour and two
    int64 sums per plan written, plan offsets read, and the order book with
    its slotting read once."""
    b = 4 * inst.order_seq.shape[0] + 4 * inst.tour_off.shape[0] + 4 * inst.plan_tour_off.shape[0]
    b += 8 * inst.n_tours + 16 * inst.n_plans
    b += 4 * inst.order_off.shape[0] + 8 * inst.n_lines
    return b


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("k_eval.cu", "wh_internal.h"):
        with open(os.path.join(ROOT, "paper_2110_13693_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, only if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "k_eval_short_midsize.json")
    try:
        with open(path) as f:
            d = json.load(f)
        if d.get("kernel_source_sha") == kernel_source_hash():
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def make_batches(n_batches, rank):
    import wh_gen
    return [wh_gen.midsize(seed=2, n_plans=PLANS_PER_STEP, plan_base=(rank * n_batches + b) * PLANS_PER_STEP)
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


# -------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2110_13693_gb300 as wh
    from paper_2110_13693_gb300 import build as whbuild

    rank, world, local = dist_env()
    assert world == args.gpus or world == 1, "--gpus must match the torchrun world size"
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group(backend="nccl", init_method="env://")
    if rank == 0 or world == 1:
        whbuild.build()
    if world > 1:
        dist.barrier()
    wh.load()
    dev = torch.device("cuda", local)

    batches = make_batches(args.batches, rank)
    lay = wh.Layout.of(batches[0].layout)
    probs = [wh.to_device(b, dev) for b in batches]
    tours = [p.n_tours for p in probs]
    costs = wh.alloc_costs(max(tours), PLANS_PER_STEP, dev)
    stream = torch.cuda.current_stream(dev)
    mask = wh.WH_ROUTE_SSHAPE | wh.WH_ROUTE_OPTIMAL

    for i in range(args.warmup):
        lay.eval_plans(probs[i % len(probs)], costs, mask, stream)
    torch.cuda.synchronize()
    assert lay.status() == 0, "device status flagged an input error"

    # ---- timed region: exactly K steps
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.15)   # let the sampler's first line land
    lay.set_timing(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    n_tours = 0
    for i in range(args.steps):
        b = i % len(probs)
        lay.eval_plans(probs[b], costs, mask, stream)
        n_tours += tours[b]
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    ktime = lay.timing()
    lay.set_timing(False)
    assert lay.status() == 0

    total_tours = n_tours
    if world > 1:
        t = torch.tensor([elapsed_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
        n = torch.tensor([n_tours], device=dev, dtype=torch.float64)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        total_tours = int(n.item())
    value = total_tours / (elapsed_ms / 1e3)

    # ---- end to end through the public API from pinned host memory
    host = []
    for b in batches:
        hp = wh.DeviceProblem(*(torch.as_tensor(getattr(b, f)).pin_memory() for f in
                                ("order_off", "line_sku", "slot_map", "plan_tour_off", "tour_off", "order_seq")),
                              b.n_sku)
        host.append(hp)
    plan_out = torch.empty((2, PLANS_PER_STEP), dtype=torch.int64).pin_memory()
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    for i in range(3):
        wh.evaluate_host(lay, host[i % len(host)], probs[i % len(probs)], costs, plan_out, mask, stream)
        stream.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e_tours, h2d, d2h = 0, 0, 0
    for i in range(e2e_steps):
        b = i % len(probs)
        hb, db = wh.evaluate_host(lay, host[b], probs[b], costs, plan_out, mask, stream)
        stream.synchronize()           # the step's plan costs are on the host now
        e_tours += tours[b]
        h2d, d2h = hb, db
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
        n = torch.tensor([e_tours], device=dev, dtype=torch.float64)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        e_tours = int(n.item())
    e2e_value = e_tours / (e2e_ms / 1e3)

    if rank != 0:
        dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel
    dom = max(ktime.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_launches, dom_ms) = dom
    per_launch_s = dom_ms / 1e3 / max(dom_launches, 1)
    alg = sum(algorithmic_bytes(b) * (args.steps // len(batches) + (1 if i < args.steps % len(batches) else 0))
              for i, b in enumerate(batches)) / args.steps
    peak, peak_kind = measured_peaks()
    achieved = alg / per_launch_s / 1e9
    traffic = recorded_traffic()
    launches = sum(v[0] for v in ktime.values())

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, ct, cp, el = cpu_oracle_rate(batches[0], args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{cp} plans ({ct} tours) of the same workload, {el:.1f} s single-threaded C"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "plans_per_step": PLANS_PER_STEP,
                   "tours_per_step": round(sum(tours) / len(tours)), "routing": "S-shape + optimal",
                   "l2": f"inputs larger than L2: {len(batches)} plan batches rotated, "
                         f"{sum(algorithmic_bytes(b) for b in batches) / 1e6:.0f} MB of step inputs (> 129 MB L2)",
                   "parallelism": f"dp{world} (independent plan batches per GPU)"},
        "plans_per_s": world * PLANS_PER_STEP * args.steps / (elapsed_ms / 1e3),
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "gpu_launches": launches,
        "kernels": {k: {"launches": v[0], "ms_total": round(v[1], 4),
                        "share": round(v[1] / max(sum(x[1] for x in ktime.values()), 1e-12), 4)}
                    for k, v in ktime.items()},
        "roofline": {"bound": "hbm", "kernel": dom_name, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": alg, "launch_ms": per_launch_s * 1e3,
                     "traffic": traffic},
        "cpu_baseline": cpu,
    }
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import wh_gen
    oracle.build()
    inst = wh_gen.midsize(seed=2, n_plans=PLANS_PER_STEP)
    # size each step so the whole run stays within about two minutes
    per_plan_s = 0.008
    plans = int(max(1, min(64, 120.0 / max(1, args.steps + args.warmup) / per_plan_s)))
    chunks = [inst.subset_plans(range(i * plans, (i + 1) * plans)) for i in range(8)]
    for i in range(args.warmup):
        oracle.eval_plans(chunks[i % len(chunks)])
    t0 = time.perf_counter()
    n = 0
    for i in range(args.steps):
        c = chunks[i % len(chunks)]
        oracle.eval_plans(c)
        n += c.n_tours
    el = time.perf_counter() - t0
    value = n / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "plans_per_step": plans,
                      "note": "each step scores a bounded sample of the same workload on the CPU oracle"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"{plans} plans per step of the same workload, single-threaded C"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
