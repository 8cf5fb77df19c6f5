"""Benchmark of the deep-copy hot path on the dense workload (3 levels, fanout
16, 273 nodes, lognormal fp32 arrays, ~338 MB), printing one JSON line.

  value  the deep copy on the default plan: dc_deep_copy (marshal into the pinned
         arena, H2D by DMA, relocation kernel) and dc_sync, host clock around
         each step; GB/s = payload bytes / step time, with its fraction of the
         measured pinned-copy H2D peak.  The input of a deep copy is the host
         structure, so the transfer is the step's work.
  device_step / roofline  the device-resident step: the arena already in HBM;
         one persistent launch relocates every pointer and runs the leaf update
         through resolved chains (dc_relocate_update), CUDA events on the
         launching stream.  roofline: algorithmic bytes (12 B per leaf element:
         read x and y, write x; 20 B per pointer slot + 16 B per block for the
         relocation) / its CUDA-event time, against the measured HBM copy peak.
         Between steps, L2 is flushed (a 512 MiB write, then a 512 MiB read of
         another buffer) unless one step streams more than twice the L2.
  e2e    through the C ABI with host buffers: deep copy + leaf update + copy back
         (into the host arrays), host clock around synchronized steps.
  batched / served  the batched workload (a forest of uneven trees in one plan
         against one plan per tree) and the request server (against sequential
         handling), each summarised; --workload batched / served print their own
         full lines.

``--impl reference`` times the CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "deep-copy GB/s vs link peak; leaf kernel HBM %; batched/served speedup, p50/p99"
NODE = "node {int32 n; int32 nchild; float* position; float* velocity; Node* child}"
WORKLOADS = {
    "dense": ("dense tree: 3 levels, fanout 16 (273 nodes), " + NODE + ", array lengths lognormal(median 65,536, "
              "sigma 1.2, cap 4,194,304), fp32 values uniform in [-1,1), seed 2"),
    "tiny": "tiny chain: 4 levels, fanout 1, " + NODE + ", 65,536 fp32 per array, seed 1",
    "deep": ("deep chain: 64 levels, fanout 1, " + NODE + ", 1,024 fp32 per interior array, 2^26 at the leaf, "
             "update through the 63-step chain to the leaf, seed 3"),
    "reloc_stress": ("pointer-heavy tree: 6 levels, fanout 16 (1,118,481 nodes), " + NODE + ", 10 fp32 per array "
                     "(the paper's n = 10 Dense case), seed 6"),
    "served": ("a Poisson stream (mean 2,000 requests/s) of deep-copy-and-update requests on node trees drawn as in "
               "the batched workload with payloads in [16 KiB, 64 MiB]; 30% of requests re-touch a tree served "
               "before (uniform over them); 40 GB HBM budget; seed 5"),
    "paper": ("the paper's own scenarios: the Linear chain {int nA; int nLnext; double* A; L* Lnext} with k = 2..10 "
              "levels of n doubles (allinit-LLused: Listing 2's scaling kernel on the last level) and the Dense tree "
              "with q = 4/8/16 structs per intermediate array, D = 3, n = 10..1000 (the Lnext[q-1] chain of Listing 2 "
              "scaled), comparing marshalling (full deep copy), pointerchain (only the effective-address array) and "
              "UVM (managed memory, first touch)"),
    "batched": ("4,096 independent node trees of uneven shape: per tree levels U{1..5}, fanout U{1..8}; array "
                "lengths lognormal(median 4,096, sigma 1.0, cap 2^20) fp32; trees redrawn until their payload is in "
                "[16 KiB, 7 MiB] (~4.4 GiB in all), seed 4"),
}


# DRAM bytes (read + write) per launch of the step's kernel from one ncu capture, by (workload, split);
# the summary beside each gives the command.  An entry stands only while the kernel is unchanged.
NCU_TRAFFIC = {
    ("dense", 128, 4): (452_980_480, "profiles/fused_kernel_dense.md"),
    ("reloc_stress", 128, 4): (196_291_200, "profiles/relocate_kernel_reloc_stress.md"),
    ("deep", 128, 4): (751_002_368, "profiles/fused_kernel_deep_batched.md"),
    ("batched", 128, 4): (7_017_168_384, "profiles/fused_kernel_deep_batched.md"),
}


def copy_check(torch, nbytes=1 << 30, reps=5):
    """A plain device-to-device copy (torch) timed in this process just before the timed steps: the
    HBM bandwidth the GPU gives right now, for comparison with the measured peak."""
    a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    best = 0.0
    for _ in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        queue_ahead(torch, 100)
        e0.record()
        b.copy_(a)
        e1.record()
        e1.synchronize()
        best = max(best, 2 * nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    del a, b
    torch.cuda.empty_cache()
    return round(best, 1)


def l2_policy(torch, step_bytes):
    """Whether to flush L2 between timed steps, and the line that says so."""
    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    if step_bytes > 2 * l2:
        return False, (f"not flushed: inputs larger than L2 (one step streams {step_bytes / 1e6:.1f} MB in the same "
                       f"order every step; L2 {l2 / 1e6:.1f} MB)")
    return True, ("flushed: 512 MiB write, then a 512 MiB read of another buffer, before every timed step "
                  "(outside the events)")


def pick_split(plan, op, args):
    """The fused step's split: --split if given (dc_set_split), else dc_autotune's pick."""
    if args.split:
        threads, ctas = (int(v) for v in args.split.split(","))
        plan.set_split(op, threads, ctas)
        return threads, ctas
    return plan.autotune(op)


def queue_ahead(torch, us: float):
    """Keep the device busy for about ``us`` microseconds, outside any events, so that the host
    has queued the launches and events that follow before the device reaches them: no timed
    region then contains host time."""
    torch.cuda._sleep(int(us * 2000))  # ~2,000 cycles per microsecond at the B300's SM clock


class L2Flush:
    """Evicts the step's data from L2 between timed steps, outside the events: a 512 MiB write,
    then a read of another 512 MiB buffer, so that a step starts with L2 holding only clean lines of
    unrelated data.  (After the write alone L2 is full of dirty lines, and the timed kernel would
    pay for writing them back.)"""

    def __init__(self, torch):
        self.torch = torch
        self.w = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
        self.r = torch.ones(128 << 20, dtype=torch.float32, device="cuda")
        self.out = torch.empty((), dtype=torch.float32, device="cuda")

    def __call__(self):
        self.w.zero_()
        self.torch.sum(self.r, dim=0, out=self.out)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def cpu_model() -> str:
    """The host CPU's model name, from /proc/cpuinfo."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or "unknown"


class Clocks:
    """nvidia-smi samples during the timed region, kept as CSV at $DC_CLOCKS_CSV (else a temp file)."""

    def __init__(self):
        self.proc = None
        self.path = os.environ.get("DC_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), f"dc_bench_clocks_{os.getpid()}.csv")

    def start(self, wait_s: float = 5.0):
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
                 "clocks.mem,temperature.gpu,temperature.memory",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
            t0 = time.time()  # the timed region starts once the sampler is producing
            while time.time() - t0 < wait_s and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        dev = int(os.environ.get("LOCAL_RANK", "0"))
        sm, mx, mem, temps, reasons = [], [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                if int(c[0]) != dev:
                    continue
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
            for lst, k in ((mem, 9), (temps, 10)):
                try:
                    lst.append(float(c[k]))
                except (ValueError, IndexError):
                    pass
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": sorted(reasons), "samples": len(sm)}
        if mem:
            out["mem_mhz"] = {"min": min(mem), "median": statistics.median(mem)}
        if temps:
            out["gpu_temp_c_max"] = max(temps)
        return out


def rank_seed(workload: str, rank: int) -> int:
    """Each rank deep-copies its own independent tree of the workload: the
    workload's seed shifted by the rank (weak scaling, no shared data)."""
    import treegen as tg
    if workload == "batched":
        return 4 + rank
    if workload == "served":
        return 5 + rank
    return tg.WORKLOADS[workload][4] + rank


def aggregate(payload_bytes: int, steps: int, t_local: float, world: int, dist=None):
    """Whole-job throughput: the bytes all ranks moved (each rank's own payload, summed) / the
    slowest rank's time.  Returns (GB/s, max time)."""
    t, total = t_local, payload_bytes
    if world > 1:
        import torch
        dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
        x = torch.tensor([t_local], dtype=torch.float64, device=dev)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
        y = torch.tensor([payload_bytes], dtype=torch.float64, device=dev)
        dist.all_reduce(y, op=dist.ReduceOp.SUM)
        total = float(y.item())
    return total * steps / t / 1e9, t


class Ranks:
    """The ranks of a torchrun job, one per GPU: a barrier, and max / sum over ranks.  With one
    rank every call is local.  The data path has no collective; these only time the job."""

    def __init__(self, torch, world: int):
        self.torch, self.world, self.dist = torch, world, None
        if world > 1:
            import torch.distributed as dist
            if not dist.is_initialized():
                dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo", init_method="env://")
            self.dist = dist

    def barrier(self):
        if self.torch.cuda.is_available():
            self.torch.cuda.synchronize()
        if self.dist:
            self.dist.barrier()

    def _reduce(self, x: float, op) -> float:
        if not self.dist:
            return x
        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = self.torch.tensor([x], dtype=self.torch.float64, device=dev)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, self.dist.ReduceOp.MAX) if self.dist else x

    def sum(self, x: float) -> float:
        return self._reduce(x, self.dist.ReduceOp.SUM) if self.dist else x

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()


def run_reference(args, rank, world):
    """The CPU oracle as it stands, one core.  Its value is the metric's first
    clause on the CPU: the oracle's deep copy alone (a recursive copy into a
    fresh host arena); the full pass (deep copy + update + copy back) is
    reported beside it.  Batched and served: the first 512 trees of the batched
    workload."""
    import oracle
    import treegen as tg
    if rank != 0:
        return
    trees = (tg.batched(512, seed=rank_seed("batched", 0)) if args.workload in ("batched", "served")
             else [tg.workload(args.workload)])
    s = trees[0].schema
    payload = sum(t.payload_bytes for t in trees)
    op = oracle_op(args.workload)
    t_copy, t_full = [], []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        copies = [oracle.deep_copy(s, t.root) for t in trees]
        t1 = time.perf_counter()
        for t, cp in zip(trees, copies):
            oracle.update(s, cp.root, op)
            oracle.copy_back(s, cp.root, t.root, op)
        t2 = time.perf_counter()
        del copies
        if i >= args.warmup:
            t_copy.append(t1 - t0)
            t_full.append(t2 - t0)
    v = payload * len(t_copy) / sum(t_copy) / 1e9
    v_full = payload * len(t_full) / sum(t_full) / 1e9
    what = "the first 512 trees of the batched workload" if len(trees) > 1 else "the whole workload"
    sample = (f"{len(t_copy)} deep copies (recursive copy into a fresh host arena) of {what} "
              f"({payload / 1e6:.1f} MB), single thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(t_copy) / len(t_copy), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "payload_bytes": payload,
                   "step": "the oracle's deep copy of the workload (or_deep_copy), one host core"},
        "cpu_baseline": {"value": round(v, 4), "unit": "GB/s", "cores": 1, "cpu_model": cpu_model(),
                         "host_cores": os.cpu_count(), "kind": "oracle", "sample": sample},
        "full_pass": {"value": round(v_full, 4), "unit": "GB/s",
                      "ms_per_step": round(1e3 * sum(t_full) / len(t_full), 3),
                      "what": "deep copy + update + copy back, the oracle's whole pass"},
        "e2e": {"value": round(v, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def oracle_op(workload):
    import oracle
    import treegen as tg
    if workload == "deep":
        return oracle.Op(sel=oracle.SEL_CHAIN, path=tg.leaf_path(64))
    return oracle.Op()


def oracle_baseline(tree, workload, budget_s=10.0):
    import oracle
    s = tree.schema
    op = oracle_op(workload)
    n, t_total = 0, 0.0
    while n < 3 or (t_total < budget_s and n < 200):
        t0 = time.perf_counter()
        cp = oracle.deep_copy(s, tree.root)
        oracle.update(s, cp.root, op)
        oracle.copy_back(s, cp.root, tree.root, op)
        t_total += time.perf_counter() - t0
        del cp
        n += 1
    v = tree.payload_bytes * n / t_total / 1e9
    return {"value": round(v, 4), "unit": "GB/s", "cores": 1, "cpu_model": cpu_model(),
            "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} full passes (deep copy + update + copy back) over the whole workload "
                      f"({tree.payload_bytes / 1e6:.1f} MB), {t_total:.1f} s on one host core"}


def cpu_update_all_cores(tree, workload, leaf_bytes, reps=5):
    """The leaf update alone on every host core (the oracle's update split into chunks over OpenMP
    threads, bit-identical to it) over the host tree in place: the CPU counterpart of the device
    step's leaf phase, with the tree already in host memory (no copy, no relocation)."""
    import oracle
    op = oracle_op(workload)
    oracle.update_parallel(tree.schema, tree.root, op)  # warm: pages and threads
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.update_parallel(tree.schema, tree.root, op)
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    return {"value": round(tree.payload_bytes / t / 1e9, 3), "unit": "GB/s", "cores": oracle.threads(),
            "cpu_model": cpu_model(), "kind": "oracle update on every host core (OpenMP)", "ms_per_step": round(t * 1e3, 3),
            "leaf_gbs": round(leaf_bytes / t / 1e9, 2),
            "sample": f"median of {reps} in-place updates of every selected array of the whole workload "
                      f"({leaf_bytes / 1e6:.1f} MB moved each)"}


def relocation_batches(torch, dc, schema, root, info, steps, barrier):
    """Mean relocate_kernel time per launch, offset records and device scan: `copies` plans of
    the same tree (each its own device arena), relocated in turn `steps` times each, back to
    back in one event pair, after warm-up; copies x the relocation's bytes moved >= 2 x L2."""
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    moved = info["reloc_table_bytes"] + 2 * info["struct_bytes"]
    copies = max(2, -(-2 * l2 // max(moved, 1)) + 1)
    if copies * info["device_bytes"] > (24 << 30):
        return None  # a tree too large to replicate in a few GB: the single-launch figures stand
    out = {}
    for name, flags in (("offset", 0), ("device_scan", dc.PLAN_DEVICE_SCAN)):
        plans = []
        for _ in range(copies):
            p = dc.Plan(schema, root, flags=flags)
            p.bind()
            p.deep_copy()
            plans.append(p)
        torch.cuda.synchronize()
        for _ in range(2):  # warm-up
            for p in plans:
                p.relocate()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        queue_ahead(torch, 1000 + 50 * steps * copies)
        e0.record()
        for _ in range(steps):
            for p in plans:
                p.relocate()
        e1.record()
        e1.synchronize()
        for p in plans:
            p.sync()
            p.destroy()
        out[name] = e0.elapsed_time(e1) * 1e-3 / (steps * copies)
    out["copies"] = copies
    return out


def pointer_heavy_relocation(torch, dc, tg, steps, warmup, flush, barrier, hbm):
    """relocate_kernel on the pointer-heavy tree (1,118,481 nodes, 2,306,867 slots in 4,370 tiles),
    offset records and device scan, for the default line: CUDA events around single launches, each
    after the L2 flush (outside the events), back-to-back launches over copies of the arena
    (relocation_batches), and one launch over a forest of four such trees.  The tree is the
    reloc_stress workload's."""
    t = tg.workload("reloc_stress")
    out = {"workload": WORKLOADS["reloc_stress"]}
    info = None
    for name, flags in (("offset", 0), ("device_scan", dc.PLAN_DEVICE_SCAN)):
        p = dc.Plan(t.schema, t.root, flags=flags)
        p.bind()
        p.deep_copy()
        p.sync()
        info = p.info
        nbytes = info["nrelocs"] * 20 + info["nblocks"] * 16
        for _ in range(warmup):
            flush()
            p.relocate()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        queue_ahead(torch, 1000 + 500 * steps)
        for e0, e1 in ev:
            flush()
            e0.record()
            p.relocate()
            e1.record()
        torch.cuda.synchronize()
        ts = [e0.elapsed_time(e1) * 1e-3 for e0, e1 in ev]
        p.sync()
        p.destroy()
        avg = statistics.mean(ts)
        out[name] = {"avg_launch_us": round(avg * 1e6, 2), "median_launch_us": round(statistics.median(ts) * 1e6, 2),
                     "achieved_gbs": round(nbytes / avg / 1e9, 1), "frac": round(nbytes / avg / 1e9 / hbm, 4)}
    out["algorithmic_bytes"] = nbytes
    out["bytes_moved"] = info["reloc_table_bytes"] + 2 * info["struct_bytes"]
    rb = relocation_batches(torch, dc, t.schema, t.root, info, steps, barrier)
    if rb:
        for name in ("offset", "device_scan"):
            out[name]["batched_us"] = round(rb[name] * 1e6, 2)
            out[name]["batched_frac"] = round(nbytes / rb[name] / 1e9 / hbm, 4)
        out["batched_copies"] = rb["copies"]
    # four such trees as one forest plan, relocated by one launch (after the flush): the kernel's
    # rate without a launch's ramp and tail per tree
    more = [tg.workload("reloc_stress", seed=100 + i) for i in range(3)]
    for name, flags in (("offset", 0), ("device_scan", dc.PLAN_DEVICE_SCAN)):
        p = dc.Plan(t.schema, [t.root] + [m.root for m in more], flags=flags)
        p.bind()
        p.deep_copy()
        p.sync()
        fbytes = p.info["nrelocs"] * 20 + p.info["nblocks"] * 16
        for _ in range(warmup):
            flush()
            p.relocate()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        queue_ahead(torch, 1000 + 500 * steps)
        for e0, e1 in ev:
            flush()
            e0.record()
            p.relocate()
            e1.record()
        torch.cuda.synchronize()
        tf = statistics.mean([e0.elapsed_time(e1) * 1e-3 for e0, e1 in ev])
        p.sync()
        p.destroy()
        out[name]["forest4_us_per_tree"] = round(tf * 1e6 / 4, 2)
        out[name]["forest4_frac"] = round(fbytes / tf / 1e9 / hbm, 4)
    for m in more:
        m.free()
    t.free()
    return out


def link_peaks(torch, nbytes=256 << 20, reps=5):
    """Pinned cudaMemcpyAsync peaks: each direction alone (best of `reps` at 256 MiB), both
    directions at once on two streams (an H2D of 2x and a D2H of 1x the bytes, the round trip's
    mix), and each direction's efficiency per size from 1 MiB to 1 GiB."""
    h = torch.empty(2 * nbytes, dtype=torch.uint8, pin_memory=True)
    h2 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(2 * nbytes, dtype=torch.uint8, device="cuda")
    d2 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = {}

    def best_of(fn, nb):
        best = 0.0
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            queue_ahead(torch, 100)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            best = max(best, nb / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        return best

    out["h2d_gbs"] = round(best_of(lambda: d[:nbytes].copy_(h[:nbytes], non_blocking=True), nbytes), 2)
    out["d2h_gbs"] = round(best_of(lambda: h[:nbytes].copy_(d[:nbytes], non_blocking=True), nbytes), 2)
    side = torch.cuda.Stream()

    def both():
        side.wait_stream(torch.cuda.current_stream())
        d.copy_(h, non_blocking=True)
        with torch.cuda.stream(side):
            h2.copy_(d2, non_blocking=True)
        torch.cuda.current_stream().wait_stream(side)

    t = 3 * nbytes / best_of(both, 3 * nbytes) / 1e9  # seconds for 2x in + 1x out
    out["bidirectional"] = {"h2d_bytes": 2 * nbytes, "d2h_bytes": nbytes, "ms": round(t * 1e3, 3),
                            "aggregate_gbs": round(3 * nbytes / t / 1e9, 2)}
    sweep = {}
    for mb in (1, 4, 16, 64, 256, 1024):
        nb = mb << 20
        hh = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
        dd = torch.empty(nb, dtype=torch.uint8, device="cuda")
        a = best_of(lambda: dd.copy_(hh, non_blocking=True), nb)
        b = best_of(lambda: hh.copy_(dd, non_blocking=True), nb)
        sweep[f"{mb}MiB"] = {"h2d_gbs": round(a, 2), "d2h_gbs": round(b, 2)}
        del hh, dd
    out["by_size"] = sweep
    # the peak is the best at 256 MiB or more
    out["h2d_gbs"] = max(out["h2d_gbs"], sweep["1024MiB"]["h2d_gbs"])
    out["d2h_gbs"] = max(out["d2h_gbs"], sweep["1024MiB"]["d2h_gbs"])
    del h, h2, d, d2
    return out


def run_batched(args, rank, world, ranks):
    out = measure_batched(args, rank, world, ranks)
    if rank == 0:
        print(json.dumps(out))


def measure_batched(args, rank, world, ranks, sample_clocks=True, cpu_sample=True):
    """One forest plan over 4,096 trees (one fused relocation + update launch;
    one round trip) against 4,096 per-structure plans (two launches each; one
    round trip each), on the same GPU.  With N ranks, 4,096 x N trees are drawn
    (sizes only) and assigned to the ranks by bytes (greedy LPT,
    dc_partition_by_bytes); each rank builds and runs its own share.  Returns
    the workload's JSON line as a dict."""
    import torch
    import treegen as tg
    import paper_1906_01128_b300 as dc
    ntrees = int(os.environ.get("DC_BATCH_TREES", "4096"))
    if world > 1:
        specs = tg.batched_specs(ntrees * world, seed=rank_seed("batched", 0))
        part, part_bytes = dc.partition_by_bytes([sp.bytes for sp in specs], world)
        trees = [sp.build() for sp, k in zip(specs, part) if k == rank]
        ntrees = len(trees)
    else:
        trees = tg.batched(ntrees, seed=rank_seed("batched", 0))
        part_bytes = [sum(t.payload_bytes for t in trees)]
    s = trees[0].schema
    payload = sum(t.payload_bytes for t in trees)
    nelem = sum(t.nelems("Node", "position") for t in trees)
    op = dc.Op()
    flush = L2Flush(torch)
    forest = dc.Plan(s, [t.root for t in trees], flags=dc.PLAN_MAP_HOST)
    forest.bind()
    info = forest.info
    forest.deep_copy()
    threads, ctas = pick_split(forest, op, args)
    forest.deep_copy()
    forest.sync()
    do_flush, l2_line = l2_policy(torch, 12 * nelem + info["nrelocs"] * 20 + info["nblocks"] * 16)
    singles = [] if args.no_compare else [dc.Plan(s, t.root, flags=dc.PLAN_MAP_HOST) for t in trees]
    for p in singles:
        p.bind()
        p.deep_copy()
        p.update(op)
    torch.cuda.synchronize()
    clocks = Clocks() if sample_clocks else None
    if clocks:
        clocks.start()

    def timed(fn, reps, label):
        """CUDA events around each step; the timed steps sit in the NVTX range ``label``."""
        for _ in range(args.warmup):
            if do_flush:
                flush()
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        queue_ahead(torch, 1000 + 500 * reps)  # the host queues every timed step meanwhile
        torch.cuda.nvtx.range_push(label)
        for e0, e1 in ev:
            if do_flush:
                flush()
            e0.record()
            fn()
            e1.record()
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        ts = [a.elapsed_time(b) * 1e-3 for a, b in ev]
        return statistics.median(ts), ts

    launches0 = dc.kernel_launches()
    ranks.barrier()
    t_forest, ts_forest = timed(lambda: forest.relocate_update(op), args.steps, "dc_step")
    ranks.barrier()
    launches = dc.kernel_launches() - launches0 - args.warmup  # the timed steps' launches (one per step)

    def per_structure():
        for p in singles:
            p.relocate()
            p.update(op)
    t_single = ranks.max(timed(per_structure, max(3, args.steps // 4), "dc_per_structure")[0]) if singles else None

    def wall(fn, reps):
        ts = []
        for i in range(args.warmup + reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            if i >= args.warmup:
                ts.append(time.perf_counter() - t0)
        return statistics.median(ts)

    ranks.barrier()
    e2e_forest = ranks.max(wall(lambda: forest.roundtrip(op), max(3, args.steps // 4)))
    e2e_single = ranks.max(wall(lambda: [p.roundtrip(op) for p in singles], 3)) if singles else None
    clk = clocks.stop() if clocks else None
    hbm, peak_kind = peaks()
    reloc_bytes = info["nrelocs"] * 20 + info["nblocks"] * 16  # 12 B entry + 8 B slot; 8 B size + 8 B offset
    fused_bytes = 12 * nelem + reloc_bytes
    t_mean = ranks.max(statistics.mean(ts_forest))  # the slowest rank's step
    t_forest = ranks.max(t_forest)
    job_payload = ranks.sum(payload)  # the bytes all ranks' steps process
    cpu = None
    if cpu_sample and not args.no_cpu and rank == 0:
        import oracle
        t_cpu, n = 0.0, 0
        for t in trees[:512]:  # a bounded sample: the first 512 trees
            t0 = time.perf_counter()
            cp = oracle.deep_copy(s, t.root)
            oracle.update(s, cp.root, oracle.Op())
            oracle.copy_back(s, cp.root, t.root, oracle.Op())
            t_cpu += time.perf_counter() - t0
            n += t.payload_bytes
        cpu = {"value": round(n / t_cpu / 1e9, 4), "unit": "GB/s", "cores": 1, "cpu_model": cpu_model(),
               "kind": "oracle",
               "sample": f"the first 512 of the {ntrees} trees ({n / 1e6:.1f} MB), deep copy + update + copy back, "
                         f"one core"}
    out = {
        "metric": METRIC, "value": round(job_payload / t_mean / 1e9, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_mean * 1e3, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["batched"], "trees": ntrees, "nodes": info["nstructs"],
                   "blocks": info["nblocks"], "payload_bytes": payload,
                   "step": "dc_relocate_update on the forest (one persistent launch)",
                   "l2": l2_line,
                   "parallelism": (f"{world} ranks, one per GPU; {len(part)} trees assigned by bytes "
                                   f"(greedy LPT), per-rank payload "
                                   f"{min(part_bytes) / 1e9:.3f}-{max(part_bytes) / 1e9:.3f} GB"
                                   if world > 1 else "1 rank")},
        "roofline": {"bound": "hbm", "kernel": "fused_kernel<float, AXPY_HALF> (relocation + leaf update)",
                     "achieved": round(fused_bytes / t_mean / 1e9, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(fused_bytes / t_mean / 1e9 / hbm, 4),
                     "traffic": NCU_TRAFFIC.get(("batched", threads, ctas), (None,))[0],
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": fused_bytes,
                     "traffic_source": NCU_TRAFFIC.get(("batched", threads, ctas), (None, None))[1],
                     "avg_launch_us": round(t_mean * 1e6, 2)},
        "batched": {"autotuned_split": {"threads_per_cta": threads, "ctas_per_sm": ctas or "max",
                                        "source": "--split" if args.split else "dc_autotune"},
                    "device_step_ms": {"forest_one_launch": round(t_forest * 1e3, 4),
                                       "per_structure_8192_launches": t_single and round(t_single * 1e3, 3)},
                    "device_speedup": t_single and round(t_single / t_forest, 2),
                    "e2e_ms": {"forest_roundtrip": round(e2e_forest * 1e3, 3),
                               "per_structure_roundtrips": e2e_single and round(e2e_single * 1e3, 3)},
                    "e2e_speedup": e2e_single and round(e2e_single / e2e_forest, 2)},
        "e2e": {"value": round(job_payload / e2e_forest / 1e9, 3), "unit": "GB/s",
                "h2d_bytes_per_step": info["data_bytes"], "d2h_bytes_per_step": 4 * nelem,
                "api": "dc_roundtrip on the forest plan, DC_PLAN_MAP_HOST"},
        "cpu_baseline": cpu, "clocks": clk, "gpu_launches": launches,
    }
    for p in singles:
        p.destroy()
    forest.destroy()
    for t in trees:
        t.free()
    return out


def run_served(args, rank, world, ranks):
    out = measure_served(args, rank, world, ranks)
    if rank == 0:
        print(json.dumps(out))


# The served stream's horizon.  A Poisson stream at 2,000 requests/s with 30% re-touches names
# 1,400 new trees per second of about 4.5 MiB each (payloads in [16 KiB, 64 MiB] as the batched
# workload draws them): ~6.6 GB of distinct host trees per second.  Every tree must exist in host
# memory before the stream starts (a request carries its tree), so the 196 GB host holds a 10 s
# stream (~66 GB of trees, ~97 GB requested with the re-touches), not the workload statement's
# 30 s (~198 GB of distinct trees).
SERVED_SECONDS = 10.0


def measure_served(args, rank, world, ranks, sample_clocks=True, duration=None):
    """The request server (8 slots, continuous batching, resident trees)
    against the same stream handled sequentially with nothing resident.
    Returns the workload's JSON line as a dict."""
    import torch
    import treegen as tg
    import paper_1906_01128_b300 as dc
    if duration is None:
        duration = float(os.environ.get("DC_SERVED_SECONDS", str(SERVED_SECONDS)))
    reqs, nkeys = tg.poisson_requests(duration, 2000.0, 0.3, seed=5 + rank)
    trees = tg.batched(nkeys, seed=5 + rank, t_min=16 << 10, t_max=64 << 20)
    s = trees[0].schema
    payload = sum(trees[k].payload_bytes for k, _, _ in reqs)
    pool = torch.empty(40 << 30, dtype=torch.uint8, device="cuda")
    pinned = int(os.environ.get("DC_SERVED_PINNED_GB", "4")) << 30  # staging for the requests in flight
    results = {}
    clocks = Clocks() if sample_clocks else None
    if clocks:
        clocks.start()
    job_payload = ranks.sum(payload)  # every rank serves its own stream
    for mode, slots, flags in (("served", 8, 0), ("sequential", 1, dc.SERVER_SEQUENTIAL)):
        srv = dc.Server(s, pool, pinned_bytes=pinned, slots=slots, flags=flags)
        ranks.barrier()
        lat = srv.run([(k, trees[k].root, a, r) for k, a, r in reqs])
        st = srv.stats
        srv.destroy()
        wall_s = ranks.max(st["wall_s"])  # the slowest rank's stream
        lat.sort()
        results[mode] = {"p50_ms": round(lat[len(lat) // 2], 3), "p99_ms": round(lat[int(len(lat) * 0.99)], 3),
                         "max_ms": round(lat[-1], 3), "wall_s": round(wall_s, 3),
                         "gbs": round(job_payload / wall_s / 1e9, 3), "resident_hits": st["resident_hits"],
                         "evictions": st["evictions"], "deep_copied_bytes": st["h2d_bytes"],
                         "copied_back_bytes": st["d2h_bytes"], "peak_resident_bytes": st["peak_resident_bytes"]}
    # capacity: the same requests all queued at once, so each mode runs as fast as it can
    saturated = {}
    for mode, slots, flags in (("served", 8, 0), ("sequential", 1, dc.SERVER_SEQUENTIAL)):
        srv = dc.Server(s, pool, pinned_bytes=pinned, slots=slots, flags=flags)
        ranks.barrier()
        srv.run([(k, trees[k].root, 0.0, r) for k, _, r in reqs])
        wall_s = ranks.max(srv.stats["wall_s"])
        srv.destroy()
        saturated[mode] = round(job_payload / wall_s / 1e9, 3)
    clk = clocks.stop() if clocks else None
    del pool
    for t in trees:
        t.free()
    sv, sq = results["served"], results["sequential"]
    out = {
        "metric": METRIC, "value": sv["gbs"], "unit": "GB/s", "n_gpus": world, "steps": len(reqs), "warmup": 0,
        "ms_per_step": round(1e3 * sv["wall_s"] / len(reqs), 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["served"], "requests": len(reqs), "distinct_trees": nkeys,
                   "duration_s": duration, "payload_bytes": payload, "slots": 8, "budget_bytes": 40 << 30},
        "served": results,
        "speedup": {"throughput": round(sv["gbs"] / sq["gbs"], 2), "p50": round(sq["p50_ms"] / sv["p50_ms"], 2),
                    "p99": round(sq["p99_ms"] / sv["p99_ms"], 2)},
        "saturated": {"served_gbs": saturated["served"], "sequential_gbs": saturated["sequential"],
                      "speedup": round(saturated["served"] / saturated["sequential"], 2),
                      "what": "the same requests all queued at time 0: the GB/s each mode sustains"},
        "e2e": {"value": sv["gbs"], "unit": "GB/s", "h2d_bytes_per_step": sv["deep_copied_bytes"] // len(reqs),
                "d2h_bytes_per_step": sv["copied_back_bytes"] // len(reqs), "api": "dc_server_run"},
        "roofline": None, "cpu_baseline": None, "clocks": clk, "gpu_launches": None,
    }
    return out


def run_paper(args, rank, world, ranks):
    """The paper's transfer-scheme comparison (Sec. 4-6) measured on this GPU:
    wall time of transfer + kernel + transfer back for marshalling (a full deep
    copy), pointerchain (only the effective-address array moves) and UVM, the
    same two schemes on a tree built in a host arena (no marshal at all), and
    the resolved vs pointer-chasing kernel time per chain length (the
    dereference cost behind Tables 3-4)."""
    import torch
    import treegen as tg
    import paper_1906_01128_b300 as dc
    n_lin = int(os.environ.get("DC_PAPER_N", str(10 ** 7)))
    reps = max(3, args.steps // 4)
    flush = L2Flush(torch)

    def wall(fn):
        ts = []
        for i in range(2 + reps):
            flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(time.perf_counter() - t0)
        return statistics.median(ts) * 1e3

    def kernel_us(fn):
        ts = []
        for i in range(2 + reps):
            flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            queue_ahead(torch, 200)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            if i >= 2:
                ts.append(e0.elapsed_time(e1) * 1e3)
        return statistics.median(ts)

    def uvm_ms(s, t, op):
        u = dc.Uvm(s, t.root)
        ts = []
        for i in range(2 + reps):
            u.prefetch(False)  # pages back on the host, as after the host initialised them
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            u.update(op)
            u.sync()
            u.copy_back()  # the host reads the result
            if i >= 2:
                ts.append(time.perf_counter() - t0)
        u.destroy()
        return statistics.median(ts) * 1e3

    def arena_ms(make, bytes_, op):
        arena = dc.HostArena(bytes_ + (64 << 20))
        t = make(arena.allocator)
        p = dc.Plan(t.schema, t.root)
        p.bind()
        full = wall(lambda: p.roundtrip(op))
        sel = wall(lambda: p.roundtrip_selected(op))
        p.destroy()
        t.free()
        arena.destroy()
        return full, sel

    ks = (2, 4, 6, 8, 10)
    # one leaf and one chase launch per k first: the launch sequence an ncu capture of the
    # dereference cost reads (-k 'leaf_kernel|chase_kernel' -c 10)
    chains = []
    for k in ks:
        t = tg.linear_tree(k, n_lin, "allinit", seed=k)
        p = dc.Plan(t.schema, t.root, flags=dc.PLAN_MAP_HOST)
        p.bind()
        op = dc.Op(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, x_field=2, scale=1.5, path=[(3, 0)] * (k - 1))
        p.deep_copy()
        p.update(op)
        p.update_chase(op)
        p.sync()
        chains.append((k, t, p, op))
    linear = []
    for k, t, p, op in chains:
        s = t.schema
        row = {"k": k, "n": n_lin, "bytes": t.payload_bytes,
               "marshalling_ms": round(wall(lambda: (p.deep_copy(), p.update(op), p.copy_back())), 3),
               "pointerchain_ms": round(wall(lambda: p.roundtrip_selected(op)), 3),
               "uvm_ms": round(uvm_ms(s, t, op), 3)}
        p.deep_copy()
        row["resolved_kernel_us"] = round(kernel_us(lambda: p.update(op)), 2)
        row["chase_kernel_us"] = round(kernel_us(lambda: p.update_chase(op)), 2)
        bytes_ = t.payload_bytes
        p.destroy()
        t.free()
        full, sel = arena_ms(lambda a: tg.linear_tree(k, n_lin, "allinit", seed=k, alloc=a), bytes_, op)
        row["arena_marshalling_ms"], row["arena_pointerchain_ms"] = round(full, 3), round(sel, 3)
        for key in ("marshalling", "pointerchain", "arena_marshalling", "arena_pointerchain"):
            row[key + "_vs_uvm"] = round(row[key + "_ms"] / row["uvm_ms"], 3)
        linear.append(row)
    dense = []
    for q in (4, 8, 16):
        for n in (10, 100, 1000):
            t = tg.dense_tree(q, n, 3, seed=q * n)
            s = t.schema
            op = dc.Op(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, type=3, x_field=1, scale=1.5, path=[(3, q - 1)] * 3)
            p = dc.Plan(s, t.root)
            p.bind()
            row = {"q": q, "n": n, "bytes": t.payload_bytes, "structs": t.nstructs,
                   "marshalling_ms": round(wall(lambda: (p.deep_copy(), p.update(op), p.copy_back())), 4),
                   "pointerchain_ms": round(wall(lambda: p.roundtrip_selected(op)), 4),
                   "uvm_ms": round(uvm_ms(s, t, op), 4)}
            bytes_ = t.payload_bytes
            p.destroy()
            t.free()
            full, sel = arena_ms(lambda a: tg.dense_tree(q, n, 3, seed=q * n, alloc=a), bytes_, op)
            row["arena_marshalling_ms"], row["arena_pointerchain_ms"] = round(full, 4), round(sel, 4)
            for key in ("pointerchain", "uvm", "arena_marshalling", "arena_pointerchain"):
                row[key + "_speedup_over_marshalling"] = round(row["marshalling_ms"] / row[key + "_ms"], 2)
            dense.append(row)
    pc = [r["pointerchain_speedup_over_marshalling"] for r in dense if r["n"] in (10, 100)]
    out = {
        "metric": METRIC, "value": round(statistics.geometric_mean(pc), 2),
        "unit": "x (Dense, n = 10 and 100: marshalling time / pointerchain time, geometric mean)",
        "n_gpus": world, "steps": reps, "warmup": 2, "ms_per_step": None, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["paper"],
                   "l2": "flushed: 512 MiB write, then a 512 MiB read of another buffer, before every timed "
                         "call (outside the timers)",
                   "linear_plan": "DC_PLAN_MAP_HOST", "dense_plan": "staged"},
        "linear_allinit_llused": linear, "dense_llused": dense,
        "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": None,
    }
    if rank == 0:
        print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="dense", choices=sorted(WORKLOADS))
    ap.add_argument("--no-compare", action="store_true", help="skip the chase / UVM comparison paths")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batched", action="store_true", help="default line: skip the batched summary")
    ap.add_argument("--no-served", action="store_true", help="default line: skip the served summary")
    ap.add_argument("--no-pointer-heavy", action="store_true",
                    help="default line: skip the relocation of the pointer-heavy tree")
    ap.add_argument("--split", default="", help="THREADS,CTAS_PER_SM for the fused step (dc_set_split) instead "
                    "of dc_autotune, e.g. 256,4: repeats a launch shape, as for an ncu capture")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "native" else args.warmup

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    import treegen as tg
    import paper_1906_01128_b300 as dc

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    ranks = Ranks(torch, world)
    if args.workload in ("batched", "served", "paper"):
        {"batched": run_batched, "served": run_served, "paper": run_paper}[args.workload](args, rank, world, ranks)
        ranks.close()
        return
    # each rank deep-copies its own independent tree (weak scaling, no data-path collective)
    tree = tg.node_tree(*tg.WORKLOADS[args.workload][:4], seed=rank_seed(args.workload, rank))
    s = tree.schema
    payload = tree.payload_bytes
    nelem = tree.nelems("Node", "position")
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plan = dc.Plan(s, tree.root)  # the walk, layout and relocation tables (host)
    t1 = time.perf_counter()
    plan.bind()  # pinned arena, transfer plan, table uploads
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    info = plan.info
    host_side = {"plan_ms": round((t1 - t0) * 1e3, 3), "bind_ms": round((t2 - t1) * 1e3, 3)}
    leaf_chain = tg.leaf_path(tg.WORKLOADS[args.workload][0])  # root -> ... -> the first leaf
    plan.resolve(leaf_chain)
    t0 = time.perf_counter()
    for _ in range(1000):
        plan.resolve(leaf_chain)
    host_side["resolve_chain_us"] = round((time.perf_counter() - t0) * 1e3, 3)  # ms for 1000 calls = us per call
    host_side["resolve_chain_steps"] = len(leaf_chain)
    if args.workload == "deep":  # only the leaf carries the long arrays: update through its chain
        op = dc.Op(sel=dc.SEL_CHAIN, path=tg.leaf_path(64))
        nelem = 1 << 26
    else:
        op = dc.Op()
    flush = L2Flush(torch)

    barrier = ranks.barrier
    max_over_ranks = ranks.max

    plan.deep_copy()
    plan.sync()
    tuned = pick_split(plan, op, args)  # the tuning runs apply the update: start again from the host tree
    plan.deep_copy()
    plan.sync()
    leaf_bytes = 12 * nelem
    # relocation: 12-byte entry read + 8-byte slot written per pointer, 8-byte size read + 8-byte offset
    # written per block; this library's relocation reads its tables and reads and writes the struct lane
    reloc_bytes = info["nrelocs"] * 20 + info["nblocks"] * 16
    reloc_moved = info["reloc_table_bytes"] + 2 * info["struct_bytes"]
    fused_bytes = leaf_bytes + reloc_bytes
    do_flush, l2_line = l2_policy(torch, fused_bytes)

    def timed_loop(parts, label):
        """CUDA events between the parts of each step (L2 policy above).  The timed steps sit
        in an NVTX range named ``label`` (an ncu capture can select them by it)."""
        for _ in range(args.warmup):
            if do_flush:
                flush()
            for f in parts:
                f()
        barrier()
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(parts) + 1)] for _ in range(args.steps)]
        # keep the device busy (outside the events) while the host queues every timed step, so
        # that no timed step waits for the host to submit it
        queue_ahead(torch, 1000 + 500 * args.steps)
        torch.cuda.nvtx.range_push(label)
        for e in ev:
            if do_flush:
                flush()  # outside the events
            e[0].record()
            for i, f in enumerate(parts):
                f()
                e[i + 1].record()
        torch.cuda.nvtx.range_pop()
        barrier()
        return [[e[i].elapsed_time(e[i + 1]) * 1e-3 for e in ev] for i in range(len(parts))]

    copy_now = copy_check(torch)
    clocks = Clocks()
    clocks.start()
    # ---- device-resident step: relocation + leaf update in one launch -------
    launches0 = dc.kernel_launches()
    (t_fused,) = timed_loop([lambda: plan.relocate_update(op)], "dc_step")
    launches = dc.kernel_launches() - launches0 - args.warmup
    plan.sync()
    value, t_step = aggregate(payload, args.steps, sum(t_fused), world, dist if world > 1 else None)
    step_median = max_over_ranks(statistics.median(t_fused))
    # the same step as two launches: each kernel on its own
    t_reloc, t_leaf = timed_loop([plan.relocate, lambda: plan.update(op)], "dc_two_launch_step")
    plan.sync()
    # the same relocation with scan records: offsets from segmented warp-shuffle prefix sums of the
    # targets' sizes on the device, one per 32-record slice
    plan_scan = dc.Plan(s, tree.root, flags=dc.PLAN_DEVICE_SCAN)
    plan_scan.bind()
    plan_scan.deep_copy()
    plan_scan.sync()
    (t_reloc_scan,) = timed_loop([plan_scan.relocate], "dc_relocate_device_scan")
    plan_scan.sync()
    plan_scan.destroy()
    del plan_scan
    # The same tree on a DC_PLAN_PACK_SMALL plan (arrays below 64 bytes at their element
    # alignment), when that shortens the arena: its device step and leaf update, same split
    packed = None
    plan_p = dc.Plan(s, tree.root, flags=dc.PLAN_PACK_SMALL)
    if plan_p.info["data_bytes"] < info["data_bytes"]:
        plan_p.bind()
        plan_p.deep_copy()
        plan_p.sync()
        plan_p.set_split(op, *tuned)
        (t_pstep,) = timed_loop([lambda: plan_p.relocate_update(op)], "dc_step_packed")
        (t_pleaf,) = timed_loop([lambda: plan_p.update(op)], "dc_leaf_packed")
        plan_p.sync()
        packed = {"plan": "DC_PLAN_PACK_SMALL", "arena_bytes": plan_p.info["data_bytes"],
                  "step_avg_us": round(statistics.mean(t_pstep) * 1e6, 2),
                  "leaf_avg_us": round(statistics.mean(t_pleaf) * 1e6, 2)}
    plan_p.destroy()
    del plan_p
    # Both relocation forms once more, as back-to-back launches over copies of the arena that
    # together stream more than twice the L2 (so no launch finds its inputs there), one event
    # pair around the batch: a launch of a few microseconds is below the event timer's
    # resolution on its own (single-launch times come in steps of about 2 us).
    reloc_batch = relocation_batches(torch, dc, s, tree.root, info, args.steps, barrier)

    # ---- the headline: the deep copy on the default plan (marshal, H2D, relocation) ----
    for _ in range(args.warmup):
        plan.deep_copy()
        plan.sync()
    barrier()
    dc_launches0 = dc.kernel_launches()
    torch.cuda.nvtx.range_push("dc_deep_copy")
    t_dc = []
    for _ in range(args.steps):
        barrier()
        t0 = time.perf_counter()
        plan.deep_copy()
        plan.sync()
        t_dc.append(time.perf_counter() - t0)
    torch.cuda.nvtx.range_pop()
    dc_launches = dc.kernel_launches() - dc_launches0
    value_dc, t_dc_total = aggregate(payload, args.steps, sum(t_dc), world, dist if world > 1 else None)

    hbm, peak_kind = peaks()
    leaf_avg = statistics.mean(t_leaf)
    reloc_avg = statistics.mean(t_reloc)
    leaf_med = statistics.median(t_leaf)
    reloc_med = statistics.median(t_reloc)
    fused_avg = statistics.mean(t_fused)
    fused_med = statistics.median(t_fused)
    pk = peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind
    roofline = {"bound": "hbm", "kernel": "fused_kernel<float, AXPY_HALF> (relocation tiles, then leaf tiles)",
                "achieved": round(fused_bytes / fused_avg / 1e9, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(fused_bytes / fused_avg / 1e9 / hbm, 4),
                "traffic": NCU_TRAFFIC.get((args.workload,) + tuple(tuned), (None,))[0], "peak_kind": pk,
                "algorithmic_bytes_per_launch": fused_bytes, "avg_launch_us": round(fused_avg * 1e6, 2),
                "median_launch_us": round(fused_med * 1e6, 2),
                "frac_at_median": round(fused_bytes / fused_med / 1e9 / hbm, 4),
                "split": {"threads_per_cta": tuned[0], "ctas_per_sm": tuned[1],
                          "source": "--split" if args.split else "dc_autotune"},
                "step_us": [round(x * 1e6, 1) for x in t_fused],
                "traffic_source": NCU_TRAFFIC.get((args.workload,) + tuple(tuned), (None, None))[1]}
    leaf_name = ("leaf_kernel<float, AXPY_HALF> (direct loads, DC_LEAF_TMA=0)" if os.environ.get("DC_LEAF_TMA") == "0"
                 else "leaf_tma_kernel<float, AXPY_HALF> (bulk copies into shared memory)")
    leaf = {"kernel": leaf_name, "algorithmic_bytes": leaf_bytes,
            "avg_launch_us": round(leaf_avg * 1e6, 2), "median_launch_us": round(leaf_med * 1e6, 2),
            "achieved_gbs": round(leaf_bytes / leaf_avg / 1e9, 1), "frac": round(leaf_bytes / leaf_avg / 1e9 / hbm, 4),
            "frac_at_median": round(leaf_bytes / leaf_med / 1e9 / hbm, 4)}

    # ---- end to end through the C ABI with host buffers ----------------------
    job_payload = ranks.sum(payload)  # every rank's own tree

    def measure_e2e(pl):
        t_e2e, t_dc, t_cb = [], [], []
        for i in range(args.warmup + max(3, args.steps // 2)):
            barrier()
            t0 = time.perf_counter()
            pl.deep_copy()
            pl.update(op)
            pl.copy_back()
            t1 = time.perf_counter()
            if i >= args.warmup:
                t_e2e.append(t1 - t0)
        for i in range(args.warmup + 5):  # deep copy alone (transfer + relocation) against the link
            barrier()
            t0 = time.perf_counter()
            pl.deep_copy()
            pl.sync()
            t1 = time.perf_counter()
            if i >= args.warmup:
                t_dc.append(t1 - t0)
        for i in range(args.warmup + 5):
            barrier()
            t0 = time.perf_counter()
            pl.copy_back()
            t1 = time.perf_counter()
            if i >= args.warmup:
                t_cb.append(t1 - t0)
        e2e_t = max_over_ranks(statistics.mean(t_e2e))
        return {"value": round(job_payload / e2e_t / 1e9, 3), "unit": "GB/s",
                "h2d_bytes_per_step": h2d_bytes(pl), "d2h_bytes_per_step": 4 * nelem,
                "ms_per_step": round(e2e_t * 1e3, 3),
                "deep_copy_gbs": round(info["data_bytes"] / statistics.median(t_dc) / 1e9, 2),
                "copy_back_gbs": round(4 * nelem / statistics.median(t_cb) / 1e9, 2)}

    def h2d_bytes(pl):  # the bytes a deep copy moves to the device: the staged spans, or the data region
        return pl.info["staging_bytes"] or pl.info["data_bytes"]

    def measure_roundtrip(pl):
        t = []
        for i in range(args.warmup + max(3, args.steps // 2)):
            barrier()
            t0 = time.perf_counter()
            pl.roundtrip(op)
            t1 = time.perf_counter()
            if i >= args.warmup:
                t.append(t1 - t0)
        tt = max_over_ranks(statistics.mean(t))
        return {"value": round(job_payload / tt / 1e9, 3), "unit": "GB/s",
                "h2d_bytes_per_step": h2d_bytes(pl), "d2h_bytes_per_step": 4 * nelem,
                "ms_per_step": round(tt * 1e3, 3)}

    e2e_staged = measure_e2e(plan)
    e2e_rt_staged = measure_roundtrip(plan)
    plan_m = dc.Plan(s, tree.root, flags=dc.PLAN_MAP_HOST)
    plan_m.bind()
    plan_m.deep_copy()
    plan_m.update(op)
    plan_m.sync()
    e2e_mapped = measure_e2e(plan_m)
    e2e_rt = measure_roundtrip(plan_m)
    plan_m.destroy()
    del plan_m
    # the same tree built in library-owned pinned memory (dc_host_arena_*: Algorithm 1's allocation
    # requests served from one buffer), so that every block is device-accessible where it lies
    arena = dc.HostArena(payload + 16 * info["nblocks"] + (1 << 20))
    tree_a = tg.node_tree(*tg.WORKLOADS[args.workload][:4], seed=rank_seed(args.workload, rank),
                          alloc=arena.allocator)
    plan_a = dc.Plan(s, tree_a.root)
    plan_a.bind()
    e2e_arena = measure_roundtrip(plan_a)
    e2e_arena["api"] = ("dc_roundtrip on the same tree built in dc_host_arena memory (the allocation-"
                        "interposing marshal: no block is marshalled or mapped per array)")
    plan_a.destroy()
    tree_a.free()
    arena.destroy()
    # the CPU baselines before the batched and served summaries: those allocate and free tens of GB
    # of host trees, after which the host's own memory runs slower for a while
    cpu = None if (args.no_cpu or rank != 0) else oracle_baseline(tree, args.workload)
    cpu_all = None if (args.no_cpu or rank != 0) else cpu_update_all_cores(tree, args.workload, leaf_bytes)
    # the default workload's relocation is a few hundred slots (launch-bound): its line also
    # carries the relocation of the pointer-heavy tree (after the headline and the CPU baselines:
    # its trees and forest take and free GB of host memory, which slows the host for a while)
    heavy = None
    if args.workload == "dense" and not args.no_pointer_heavy:
        heavy = pointer_heavy_relocation(torch, dc, tg, args.steps, args.warmup, flush, barrier, peaks()[0])
    batched = served = None
    if not args.no_batched:
        bo = measure_batched(args, rank, world, ranks, sample_clocks=False, cpu_sample=False)
        bb = bo["batched"]
        batched = {"workload": bo["config"]["workload"], "trees": bo["config"]["trees"],
                   "payload_bytes": bo["config"]["payload_bytes"],
                   "device_step_ms": bb["device_step_ms"], "device_speedup": bb["device_speedup"],
                   "device_step_gbs": bo["value"], "device_step_frac_of_hbm": bo["roofline"]["frac"],
                   "e2e_ms": bb["e2e_ms"], "e2e_speedup": bb["e2e_speedup"], "e2e_gbs": bo["e2e"]["value"],
                   "split": bb["autotuned_split"],
                   "what": "one forest plan (one persistent relocation + update launch; one round trip) "
                           "against one plan per tree (two launches each; one round trip each)"}
    if not args.no_served:
        so = measure_served(args, rank, world, ranks, sample_clocks=False)
        served = {"workload": so["config"]["workload"], "duration_s": so["config"]["duration_s"],
                  "requests": so["config"]["requests"], "distinct_trees": so["config"]["distinct_trees"],
                  "payload_bytes": so["config"]["payload_bytes"], "slots": so["config"]["slots"],
                  "served": so["served"]["served"], "sequential": so["served"]["sequential"],
                  "speedup": so["speedup"], "saturated": so["saturated"],
                  "horizon": f"{SERVED_SECONDS:g} s: the host memory holds every distinct tree of a "
                             f"{SERVED_SECONDS:g} s stream, not of 30 s"}
    clk = clocks.stop()
    # the fastest public path end to end: dc_roundtrip or the three calls, on a mapped or the default plan
    e2e_staged_calls = {k: v for k, v in e2e_staged.items() if k not in ("deep_copy_gbs", "copy_back_gbs")}
    candidates = [
        (e2e_rt, "dc_roundtrip (deep copy + leaf update + copy back in one call), plan flag DC_PLAN_MAP_HOST"),
        (e2e_mapped, "dc_deep_copy + dc_update_leaves + dc_copy_back, plan flag DC_PLAN_MAP_HOST"),
        (e2e_rt_staged, "dc_roundtrip on the default plan (staged" +
         (", by host spans" if info["staging_bytes"] else "") + ")"),
        (e2e_staged_calls, "dc_deep_copy + dc_update_leaves + dc_copy_back on the default plan"),
    ]
    best, api = max(candidates, key=lambda c: c[0]["value"])
    e2e = dict(best)
    e2e["api"] = api
    link = link_peaks(torch)
    for mode, r in (("staged", e2e_staged), ("map_host", e2e_mapped)):
        link[f"deep_copy_frac_of_h2d_peak_{mode}"] = round(r["deep_copy_gbs"] / link["h2d_gbs"], 4)
        link[f"copy_back_frac_of_d2h_peak_{mode}"] = round(r["copy_back_gbs"] / link["d2h_gbs"], 4)
    # the round trip moves both directions at once: against the two copy engines' aggregate
    rt_bytes = e2e_rt["h2d_bytes_per_step"] + e2e_rt["d2h_bytes_per_step"]
    link["roundtrip_link_gbs"] = round(rt_bytes / (e2e_rt["ms_per_step"] * 1e-3) / 1e9, 2)
    link["roundtrip_frac_of_bidirectional_peak"] = round(link["roundtrip_link_gbs"] /
                                                         link["bidirectional"]["aggregate_gbs"], 4)
    link["roundtrip_host_arena_frac_of_bidirectional_peak"] = round(
        rt_bytes / (e2e_arena["ms_per_step"] * 1e-3) / 1e9 / link["bidirectional"]["aggregate_gbs"], 4)

    # ---- comparison paths (same GPU) -----------------------------------------
    compare = None
    if not args.no_compare and rank == 0:
        compare = {}
        t = []
        for i in range(5):
            if do_flush:
                flush()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            queue_ahead(torch, 200)
            e0.record()
            plan.update_chase(op)
            e1.record()
            e1.synchronize()
            if i:
                t.append(e0.elapsed_time(e1))
        compare["chase_kernel_us"] = round(1e3 * statistics.mean(t), 2)
        compare["resolved_leaf_kernel_us"] = round(leaf_avg * 1e6, 2)
        u = dc.Uvm(s, tree.root)
        first, pref = [], []
        for i in range(3):
            u.prefetch(False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            queue_ahead(torch, 200)
            e0.record()
            u.update(op)
            e1.record()
            e1.synchronize()
            first.append(e0.elapsed_time(e1))
            u.prefetch(True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            queue_ahead(torch, 200)
            e0.record()
            u.update(op)
            e1.record()
            e1.synchronize()
            pref.append(e0.elapsed_time(e1))
        compare["uvm_first_touch_kernel_ms"] = round(statistics.median(first), 3)
        compare["uvm_prefetched_kernel_ms"] = round(statistics.median(pref), 3)
        u.destroy()


    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value_dc, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * t_dc_total / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "nodes": info["nstructs"], "blocks": info["nblocks"],
                       "payload_bytes": payload, "arena_bytes": info["data_bytes"], "elements": nelem,
                       "step": "dc_deep_copy + dc_sync on the default plan (marshal into the pinned arena, H2D "
                               "by DMA in chunks, relocation kernel), host clock; the tree is in host memory "
                               "when a step starts",
                       "l2": "the deep copy's inputs are in host memory; " + l2_line + " for the device step",
                       "parallelism": f"{world} independent tree(s), one per GPU"},
            "deep_copy": {"gbs": round(value_dc, 3), "h2d_bytes_per_step": info["staging_bytes"] or info["data_bytes"],
                          "frac_of_h2d_peak": round(value_dc / link["h2d_gbs"], 4),
                          "median_ms": round(1e3 * statistics.median(t_dc), 3),
                          "step_ms": [round(1e3 * x, 3) for x in t_dc],
                          "plan": ("default (staged by host spans: streaming copies of the tree's host spans, "
                                   "DMA per chunk, blocks placed by one device launch)" if info["staging_bytes"] else
                                   "default (staged: marshal by host threads, DMA per chunk)"),
                          "map_host_gbs": e2e_mapped["deep_copy_gbs"],
                          "map_host_frac_of_h2d_peak": round(e2e_mapped["deep_copy_gbs"] / link["h2d_gbs"], 4)},
            "device_step": {"value": round(value, 2), "unit": "GB/s", "ms_per_step": round(1e3 * t_step / args.steps, 4),
                            "step": "dc_relocate_update (relocation + leaf update, one persistent launch, split by "
                                    "dc_autotune) on the resident arena, CUDA events",
                            "gpu_launches": launches},
            "roofline": roofline,
            "leaf": leaf,
            "relocation": {"kernel": "relocate_kernel", "avg_launch_us": round(reloc_avg * 1e6, 2),
                           "median_launch_us": round(reloc_med * 1e6, 2),
                           "algorithmic_bytes": reloc_bytes, "achieved_gbs": round(reloc_bytes / reloc_avg / 1e9, 1),
                           "frac": round(reloc_bytes / reloc_avg / 1e9 / hbm, 4), "bytes_moved": reloc_moved,
                           **({"batched_us": round(reloc_batch["offset"] * 1e6, 2),
                               "batched_frac": round(reloc_bytes / reloc_batch["offset"] / 1e9 / hbm, 4),
                               "batched_copies": reloc_batch["copies"]} if reloc_batch else {})},
            "relocation_device_scan": {
                "kernel": "relocate_kernel, DC_PLAN_DEVICE_SCAN (offsets from segmented warp prefix sums of the targets' sizes, one per 32-record slice seeded with its first offset)",
                "avg_launch_us": round(statistics.mean(t_reloc_scan) * 1e6, 2),
                "median_launch_us": round(statistics.median(t_reloc_scan) * 1e6, 2),
                "frac": round(reloc_bytes / statistics.mean(t_reloc_scan) / 1e9 / hbm, 4),
                **({"batched_us": round(reloc_batch["device_scan"] * 1e6, 2),
                    "batched_frac": round(reloc_bytes / reloc_batch["device_scan"] / 1e9 / hbm, 4)}
                   if reloc_batch else {})},
            "relocation_pointer_heavy": heavy,
            "packed": packed and {**packed,
                                  "step_frac": round(fused_bytes / (packed["step_avg_us"] * 1e-6) / 1e9 / hbm, 4),
                                  "leaf_frac": round(leaf_bytes / (packed["leaf_avg_us"] * 1e-6) / 1e9 / hbm, 4)},
            "two_launch_step_us": round((reloc_avg + leaf_avg) * 1e6, 2),
            "step_median_ms": round(step_median * 1e3, 4),
            "hbm_copy_gbs_now": copy_now,
            "host_side": host_side,
            "e2e": e2e, "e2e_three_calls_map_host": e2e_mapped, "e2e_staged": e2e_staged,
            "e2e_roundtrip_staged": e2e_rt_staged,
            "e2e_host_arena": e2e_arena, "link": link, "compare": compare, "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
            "batched": batched, "served": served,
            "clocks": clk,
            "gpu_launches": dc_launches,
        }
        print(json.dumps(out))
    plan.destroy()
    ranks.close()


if __name__ == "__main__":
    main()
