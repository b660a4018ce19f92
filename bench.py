#!/usr/bin/env python
"""Benchmark of the Louvain hot path on GB300: M edges/s = |E| / total time.

One step = one whole ``louvain_run`` (every pass of local moving and
aggregation plus the final modularity) on a graph already resident in HBM.
|E| counts both directions of every edge (directed CSR entries), as the
paper's Table 2 does.  Default workload: R-MAT scale 27, edge factor 16,
(a, b, c) = (0.57, 0.19, 0.19), seed 13, unit weights (synthetic; 134M
vertices, 4.2 billion entries), timed in the plain form (`value`) and in the
learned-skip form (`learned_skip`) on the same graph and launch schedule.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the same
workload on its own GPU (the single-graph method has no shardable exchange);
the value is the sum of edges over ranks divided by the slowest rank's time.
``--impl reference`` times the CPU oracle (the plain restatement of the
paper's algorithms) on the host cores on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2501_19004_gb300 import graphgen as gg  # noqa: E402

METRIC = "Louvain M edges/s (|E|/total time), plain vs learned-skip at ΔQ≤1e-3"
UNIT = "M edges/s"

WORKLOADS = {
    "rmat24": dict(kind="rmat", scale=24, ef=16, seed=7, desc="R-MAT scale 24, edge factor 16, "
                   "(a,b,c,d)=(0.57,0.19,0.19,0.05), symmetrised, deduplicated, no self-loops, unit int32 weights, "
                   "int32 ids / int64 offsets, seed 7"),
    "grid8192": dict(kind="grid", side=8192, frac=0.02, seed=11, desc="8192x8192 4-neighbour grid + 2% random "
                     "long-range edges, uniform integer weights 1-8, seed 11"),
    "grid4096": dict(kind="grid", side=4096, frac=0.02, seed=11, desc="4096x4096 4-neighbour grid + 2% random "
                     "long-range edges, uniform integer weights 1-8, seed 11 (profiling case: the grid workload's "
                     "generator at a quarter of the size)"),
    "sbm1000": dict(kind="sbm", n=1000, block=100, p_in=0.1, p_out=0.002, seed=1, desc="planted-partition SBM, "
                    "1,000 vertices in 10 blocks of 100, p_in=0.1, p_out=0.002, seed 1"),
    "rmat22": dict(kind="rmat", scale=22, ef=16, seed=7, desc="R-MAT scale 22, edge factor 16, "
                   "(a,b,c,d)=(0.57,0.19,0.19,0.05), symmetrised, deduplicated, no self-loops, unit int32 weights, "
                   "seed 7 (profiling case: the default workload's generator at a quarter of the size)"),
    "rmat27": dict(kind="rmat", scale=27, ef=16, seed=13, desc="R-MAT scale 27, edge factor 16, "
                   "(a,b,c,d)=(0.57,0.19,0.19,0.05), symmetrised, deduplicated, no self-loops, unit int32 weights, "
                   "seed 13 (learned-skip evaluation graph)"),
    "bsbm4096": dict(kind="batch", G=4096, first=0, desc="batch of 4,096 planted-partition SBM graphs, vertex "
                     "counts log-uniform in 200-200,000, mean degree uniform in 8-32, blocks of 50, mixing ratio "
                     "uniform in 0.1-0.4, unit int32 weights, seeds 0-4095, one batched context"),
}
# bounded CPU-oracle samples: the same generator at a smaller size.  The
# CPU-baseline leg of a GPU run times one oracle run of SAMPLES; the reference
# arm times one oracle run of REF_SAMPLES per step.
REF_SAMPLES = {
    "rmat24": dict(kind="rmat", scale=20, ef=16, seed=7, desc="R-MAT scale 20 (same generator and parameters)"),
    "grid8192": dict(kind="grid", side=1024, frac=0.02, seed=11, desc="1024x1024 grid (same generator)"),
    "grid4096": dict(kind="grid", side=1024, frac=0.02, seed=11, desc="1024x1024 grid (same generator)"),
    "sbm1000": dict(kind="sbm", n=1000, block=100, p_in=0.1, p_out=0.002, seed=1, desc="the full workload"),
    "rmat22": dict(kind="rmat", scale=20, ef=16, seed=7, desc="R-MAT scale 20 (same generator and parameters)"),
    "rmat27": dict(kind="rmat", scale=20, ef=16, seed=13, desc="R-MAT scale 20 (same generator and parameters)"),
    "bsbm4096": dict(kind="batch", G=48, first=0, desc="graphs 0-47 of the batch, one oracle run each"),
}
SAMPLES = {
    "rmat24": dict(kind="rmat", scale=21, ef=16, seed=7, desc="R-MAT scale 21 (same generator and parameters)"),
    "grid8192": dict(kind="grid", side=1448, frac=0.02, seed=11, desc="1448x1448 grid (same generator)"),
    "grid4096": dict(kind="grid", side=1024, frac=0.02, seed=11, desc="1024x1024 grid (same generator)"),
    "sbm1000": dict(kind="sbm", n=1000, block=100, p_in=0.1, p_out=0.002, seed=1, desc="the full workload"),
    "rmat22": dict(kind="rmat", scale=20, ef=16, seed=7, desc="R-MAT scale 20 (same generator and parameters)"),
    "rmat27": dict(kind="rmat", scale=21, ef=16, seed=13, desc="R-MAT scale 21 (same generator and parameters)"),
    "bsbm4096": dict(kind="batch", G=256, first=0, desc="graphs 0-255 of the batch, one oracle run each"),
}


# timing groups that are one kernel per launch (candidates for the roofline)
SINGLE_KERNELS = {"select", "move_thread", "move_group", "move_half", "move_wide", "move_warp", "move_mid", "move_block", "move_hub", "apply",
                  "pass_init", "merge_thread", "merge_warp", "merge_mid", "merge_block", "merge_big", "merge_xl", "merge_group",
                  "dendrogram"}


def make_graph(w):
    """The workload's graph; for a batch, (union CSR, vertex offsets)."""
    if w["kind"] == "batch":
        return gg.batched_sbm_union(w["G"], w.get("first", 0))
    if w["kind"] == "rmat":
        return gg.rmat(w["scale"], w["ef"], seed=w["seed"])
    if w["kind"] == "grid":
        return gg.grid(w["side"], w["frac"], seed=w["seed"])
    return gg.sbm(w["n"], w["block"], w["p_in"], w["p_out"], seed=w["seed"])


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def sample_graphs(w):
    """(list of graphs, total entries) of a CPU-oracle sample."""
    if w["kind"] == "batch":
        gs = [gg.batched_sbm(k) for k in range(w.get("first", 0), w.get("first", 0) + w["G"])]
    else:
        gs = [make_graph(w)]
    return gs, sum(x.nnz for x in gs)


def oracle_steps(gs, steps: int, warmup: int):
    import oracle
    cfg = oracle.Config()
    for _ in range(warmup):
        for g in gs:
            oracle.louvain(g, cfg)
    t0 = time.perf_counter()
    for _ in range(steps):
        for g in gs:
            oracle.louvain(g, cfg)
    dt = time.perf_counter() - t0
    return dt, oracle.num_threads()


def move_bin_degrees(kernel: str, sched: dict):
    """Degree range [lo, hi] (hi None: unbounded) of the vertices a
    local-moving kernel takes under a launch schedule; None for kernels that
    are not a degree bin of local moving."""
    gm, hm, wm = sched["group_max"], sched["half_max"], sched["warp_max"]
    return {"move_thread": [1, 16], "move_group": [17, gm], "move_half": [gm + 1, hm], "move_warp": [hm + 1, wm],
            "move_mid": [wm + 1, 1024], "move_block": [1025, 4096], "move_wide": [4097, 32768],
            "move_hub": [32769, None]}.get(kernel)


def _fmix32(h):
    """MurmurHash3's 32-bit finaliser on a numpy uint32 array."""
    h = h.astype(np.uint64)
    m = np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x85EBCA6B)) & m
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0xC2B2AE35)) & m
    h ^= h >> np.uint64(16)
    return h


def first_launch_entries(g, kernel: str, sched: dict, launches: int, buckets: int = 4, seed: int = 0):
    """Row entries that the first `launches` launches of a local-moving bin
    kernel take in a plain run: the buckets 0, 1, ... of iteration 0 of pass
    0, where every vertex is unprocessed (bucket hash as in
    include/louvain.h).  Used to turn the DRAM bytes of an ncu capture of
    those launches into bytes per entry."""
    lo, hi = move_bin_degrees(kernel, sched)
    deg = np.diff(g.offsets)
    inbin = (deg >= lo) & ((deg <= hi) if hi is not None else True)
    fold = (seed & 0xFFFFFFFF) ^ (seed >> 32)
    salt = int(_fmix32(np.array([fold ^ ((0 * 0x9E3779B1) & 0xFFFFFFFF)], dtype=np.uint64))[0])
    b = _fmix32(np.arange(g.n, dtype=np.uint64) ^ np.uint64(salt)) % np.uint64(buckets)
    return [int(deg[inbin & (b == np.uint64(k))].sum()) for k in range(launches)]


def stored_traffic(kernel: str):
    """(DRAM bytes per row entry, capture record) of `kernel` from
    profiles/traffic.json, or (None, None) if there is none or the library's
    sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        tj = json.load(open(path))
    except (OSError, ValueError):
        return None, None
    ent = tj.get(kernel)
    if not ent or ent.get("sources") != source_hash(kernel_sources(kernel)):
        return None, None
    return ent.get("dram_bytes_per_entry"), ent


def kernel_sources(kernel: str):
    """The CUDA source files whose code a kernel group runs: its own
    translation unit and every header (the hub path lives in big.cu, the
    aggregation kernels in aggr.cu, local moving in move.cu)."""
    tu = ("big.cu" if kernel in ("move_hub", "move_hub_eval", "merge_big", "merge_big_emit")
          else "move.cu" if kernel.startswith("move_") or kernel in ("select", "apply", "pass_init", "mlp_select")
          else "aggr.cu")
    headers = [f for f in os.listdir(os.path.join(ROOT, "paper_2501_19004_gb300", "csrc")) if f.endswith((".cuh", ".h"))]
    return [tu] + headers


def source_hash(files=None) -> str:
    """FNV-1a of the library's CUDA sources (all of them, or the named files
    of the source folder), so that a stored capture is used only for the
    kernels it measured."""
    import glob
    h = 0xcbf29ce484222325
    csrc = os.path.join(ROOT, "paper_2501_19004_gb300", "csrc")
    paths = glob.glob(os.path.join(csrc, "*")) if files is None else [os.path.join(csrc, f) for f in files]
    for f in sorted(paths):
        for byte in open(f, "rb").read():
            h = ((h ^ byte) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return f"{h:016x}"


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest x over all ranks (the slowest rank's time), by one
    all-reduce; x itself on a single rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, steps: int, world: int, seconds: float) -> float:
    """Whole-job M units/s: every rank processed units_per_rank in each of
    `steps` steps, and the job took as long as its slowest rank."""
    return units_per_rank * steps * world / seconds / 1e6


def run_reference(args, wname):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sample = REF_SAMPLES[wname]
    gs, nnz = sample_graphs(sample)
    dt, cores = oracle_steps(gs, args.steps, args.warmup)
    value = nnz * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": WORKLOADS[wname]["desc"], "sample": sample["desc"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample['desc']}: {nnz} entries, whole run per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat27", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-skip leg")
    ap.add_argument("--no-async", action="store_true", help="skip the asynchronous-form leg")
    ap.add_argument("--no-leiden", action="store_true", help="skip the Leiden-form leg")
    ap.add_argument("--skip-threshold", type=float, default=None, help="default: the stored model's setting")
    ap.add_argument("--learned-min-degree", type=int, default=None, help="default: the stored model's setting")
    ap.add_argument("--graphs", type=int, default=0, help="batch workloads: run only the first N graphs")
    ap.add_argument("--batch-leg", type=int, default=4096,
                    help="single-graph workloads: also time the batched workload on its first N graphs (0: no leg)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch schedule")
    ap.add_argument("--autotune-runs", type=int, default=32)
    ap.add_argument("--sequential-sample", type=int, default=256,
                    help="batch workloads: graphs run one context at a time for comparison")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args, args.workload)

    import torch
    import torch.distributed as dist
    from paper_2501_19004_gb300 import louvain as lv

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if world > 1:
            dist.barrier()

    w = dict(WORKLOADS[args.workload])
    batch = w["kind"] == "batch"
    if batch and args.graphs:
        w["G"] = args.graphs
        w["desc"] += f" (first {args.graphs} graphs only)"
    vo = None
    if batch:
        g, vo = make_graph(w)
    else:
        g = make_graph(w)
    dg = lv.DeviceCSR.from_host(g, dev)
    torch.cuda.synchronize()

    sched = None  # the tuned launch schedule, applied to every context below

    def new_ctx(graph, cfg=None):
        c = lv.LouvainBatch(graph, vo, cfg) if batch else lv.Louvain(graph, cfg)
        if sched:
            c.set_schedule(sched)
        return c

    all_mask = (1 << len(lv.KERNELS)) - 1
    ctx = new_ctx(dg, lv.Config(profile_mask=all_mask))
    # the library's autotuner picks the launch schedule on this workload
    # (timed runs before the measurement; results do not depend on it)
    tune = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        rep = ctx.autotune(args.autotune_runs)
        sched = ctx.schedule()
        tune = {"seconds": round(time.perf_counter() - t0, 2), "runs": rep["runs"], "start_ms": rep["start_ms"],
                "tuned_ms": rep["tuned_ms"], "schedule": sched}
    # warm-up 1: every kernel group timed, to find the dominant kernel; the
    # bins run one after another here (with concurrent bins, a kernel's event
    # time would include the others running beside it)
    run_sched = ctx.schedule()
    serial_sched = dict(run_sched, concurrent=0)
    ctx.set_schedule(serial_sched)
    ctx.run()
    prof = ctx.stats()["kernels"]
    dom = max((k for k in prof if prof[k]["launches"] > 0 and k in SINGLE_KERNELS), key=lambda k: prof[k]["ms"])
    ctx.set_schedule(run_sched)
    ctx.set_profile(lv.kernel_mask(dom))
    for _ in range(args.warmup - 1):
        ctx.run()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    dom_ms = dom_bytes = 0.0
    dom_launches = launches = 0
    e0.record(stream)
    for _ in range(args.steps):
        ctx.run()
        st = ctx.stats()
        dom_ms += st["kernels"][dom]["ms"]
        dom_bytes += st["kernels"][dom]["bytes"]
        dom_launches += st["kernels"][dom]["launches"]
        launches += st["kernel_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, world, dev)
    res = ctx.result()
    st = ctx.stats()
    value = job_rate(g.nnz, args.steps, world, ms / 1e3)
    # the dominant kernel once more with the bins serialised (untimed run)
    serial = None
    if run_sched.get("concurrent"):
        ctx.set_schedule(serial_sched)
        ctx.run()
        k = ctx.stats()["kernels"][dom]
        ctx.set_schedule(run_sched)
        if k["ms"] > 0:
            serial = {"achieved": k["bytes"] / (k["ms"] / 1e3) / 1e9, "avg_launch_ms": k["ms"] / max(k["launches"], 1),
                      "launches": k["launches"]}

    # end to end through the public API from pinned host memory
    e2e = None
    if args.e2e_steps > 0:
        off_p = torch.from_numpy(g.offsets).pin_memory()
        col_p = torch.from_numpy(g.cols).pin_memory()
        host = gg.CSR(off_p.numpy(), col_p.numpy(), None)
        memb_p = torch.empty(g.n, dtype=torch.int32).pin_memory()
        ctx.close()
        with new_ctx(host) as c2:  # warm the allocator pool
            c2.run()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            with new_ctx(host) as c2:
                c2.run()
                lv.louvain_memberships(c2.ctx, memb_p.numpy())
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_rate(g.nnz, args.e2e_steps, world, dt), "unit": UNIT,
               "h2d_bytes_per_step": int(g.offsets.nbytes + g.cols.nbytes),
               "d2h_bytes_per_step": int(g.n * 4), "steps": args.e2e_steps}
    else:
        ctx.close()

    # learned-skip leg: the same workload and step count with the predictor
    learned = None
    if batch:
        summary = {"modularity_mean": float(np.mean(res.modularity)), "communities": int(res.summary[:, 1].sum()),
                   "passes_max": int(res.summary[:, 0].max()), "graphs": int(vo.shape[0] - 1)}
    else:
        summary = {"modularity": res.modularity, "communities": res.communities, "passes": res.passes}
    def timed_leg(cfg):
        """Warm-up and timed runs of another configuration on the same graph
        and schedule; returns (ms for all timed steps, result, stats)."""
        c = lv.Louvain(dg, cfg)
        if sched:
            c.set_schedule(sched)
        for _ in range(args.warmup):
            c.run()
        torch.cuda.synchronize()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            c.run()
        e1.record(stream)
        torch.cuda.synchronize()
        t_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
        r, s_ = c.result(), c.stats()
        c.close()
        return t_ms, r, s_

    if not args.no_learned and not batch:
        from paper_2501_19004_gb300 import predictor
        model = predictor.load_default()
        source = "stored model (R-MAT 20-22 traces)"
        if model is None:
            model, _ = predictor.train_default()
            source = "trained in this run (R-MAT 20-22 traces)"
        over = {}
        if args.skip_threshold is not None:
            over["skip_threshold"] = args.skip_threshold
        if args.learned_min_degree is not None:
            over["learned_min_degree"] = args.learned_min_degree
        lcfg = predictor.default_config(model, **over)
        lms, lres, lst = timed_leg(lcfg)
        learned = {"value": job_rate(g.nnz, args.steps, world, lms / 1e3), "unit": UNIT,
                   "ms_per_step": lms / args.steps, "modularity": lres.modularity,
                   "dq_vs_plain": lres.modularity - res.modularity, "skip_threshold": lcfg.skip_threshold,
                   "min_degree": lcfg.learned_min_degree, "fallback": lcfg.learned_fallback,
                   "skip_clears": lcfg.learned_skip_clears,
                   "evaluated": lst["evaluated"], "evaluated_plain": st["evaluated"], "skipped": lst["skipped"],
                   "passes": lres.passes, "learned_passes": lst.get("learned_passes"), "model": source,
                   "speedup_vs_plain": (lms and ms / lms)}

    # asynchronous form (moves applied at their decision; not reproducible)
    asynchronous = None
    if not args.no_async and not batch:
        ams, ares, ast = timed_leg(lv.Config(asynchronous=True))
        asynchronous = {"value": job_rate(g.nnz, args.steps, world, ams / 1e3), "unit": UNIT,
                        "ms_per_step": ams / args.steps, "modularity": ares.modularity,
                        "dq_vs_plain": ares.modularity - res.modularity, "passes": ares.passes,
                        "iterations": ast["iterations"], "evaluated": ast["evaluated"],
                        "evaluated_plain": st["evaluated"], "communities": ares.communities}

    # the Leiden form (refinement before aggregation; deterministic)
    leiden = None
    if not args.no_leiden and not batch:
        rms, rres, rst = timed_leg(lv.Config(refine=True))
        leiden = {"value": job_rate(g.nnz, args.steps, world, rms / 1e3), "unit": UNIT,
                  "ms_per_step": rms / args.steps, "modularity": rres.modularity,
                  "dq_vs_plain": rres.modularity - res.modularity, "passes": rres.passes,
                  "communities": rres.communities, "exit_reason": rres.exit_reason}

    peaks, src = load_peaks()
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else None
    # DRAM bytes per launch: a small capture's bytes per row entry (ncu on
    # R-MAT scale 22, profiles/traffic.json, current sources only) times the
    # entries of this run's average launch of the dominant kernel
    traffic = None
    per_entry, tent = stored_traffic(dom)
    dom_entries = st["kernels"].get(dom, {}).get("entries", 0.0)
    if per_entry and dom_launches:
        traffic = per_entry * (dom_entries * args.steps) / dom_launches
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": (achieved / peaks["hbm_gbs"]) if achieved else None, "peak_source": f"{src} hbm_gbs",
                "traffic": traffic,
                "algorithmic_bytes_per_launch": dom_bytes / max(dom_launches, 1),
                "avg_launch_ms": dom_ms / max(dom_launches, 1), "launches": dom_launches,
                "concurrent_bins": bool(run_sched.get("concurrent"))}
    if serial:
        serial["frac"] = serial["achieved"] / peaks["hbm_gbs"]
        roofline["serial"] = serial
    # whole run: every kernel's algorithmic bytes of the last timed run at
    # the peak give the shortest possible run and so a bound on edges/s
    run_bytes = sum(float(v.get("bytes", 0.0)) for v in st.get("kernels", {}).values())
    if run_bytes > 0:
        bound_ms = run_bytes / (peaks["hbm_gbs"] * 1e9) * 1e3
        roofline["run"] = {"algorithmic_bytes": run_bytes, "bound_ms": bound_ms,
                           "implied_bound": job_rate(g.nnz, 1, world, bound_ms / 1e3),
                           "frac": bound_ms / (ms / args.steps)}

    # batch only: the same graphs one context at a time (a strided sample),
    # the way a single-graph library would run them
    sequential = None
    if batch and args.sequential_sample > 0:
        G = int(vo.shape[0] - 1)
        stride = max(1, G // args.sequential_sample)
        picks = list(range(0, G, stride))[:args.sequential_sample]
        seq_ms = 0.0
        seq_nnz = 0
        for k in picks:
            a, b = int(vo[k]), int(vo[k + 1])
            ea, eb = int(g.offsets[a]), int(g.offsets[b])
            sub_g = lv.DeviceCSR((dg.offsets[a:b + 1] - ea).contiguous(), (dg.cols[ea:eb] - a).contiguous())
            with lv.Louvain(sub_g) as c1:
                if sched:
                    c1.set_schedule(sched)
                c1.run()
                s0 = torch.cuda.Event(enable_timing=True)
                s1 = torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                c1.run()
                s1.record(stream)
                torch.cuda.synchronize()
                seq_ms += s0.elapsed_time(s1)
            seq_nnz += sub_g.nnz
        sequential = {"value": seq_nnz / (seq_ms / 1e3) / 1e6, "unit": UNIT, "graphs": len(picks),
                      "stride": stride, "ms_total": seq_ms,
                      "note": "each sampled graph in its own context, one louvain_run each"}

    # the batched workload as an extra leg beside a single-graph workload: one
    # context over the first N graphs of the 4,096-graph planted-partition
    # batch, default schedule with concurrent bins, timed like the main leg
    batch_leg = None
    if not batch and args.batch_leg > 0:
        del dg
        torch.cuda.empty_cache()
        wb = dict(WORKLOADS["bsbm4096"], G=min(args.batch_leg, 4096))
        ub, vob = make_graph(wb)
        dub = lv.DeviceCSR.from_host(ub, dev)
        with lv.LouvainBatch(dub, vob) as cb:
            cb.set_schedule(dict(concurrent=1))
            for _ in range(max(args.warmup, 1)):
                cb.run()
            torch.cuda.synchronize()
            barrier()
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            for _ in range(args.steps):
                cb.run()
            b1.record(stream)
            torch.cuda.synchronize()
            bms = max_over_ranks(b0.elapsed_time(b1), world, dev)
            bst = cb.stats()
        batch_leg = {"workload": wb["desc"] + (f" (first {wb['G']} graphs)" if wb["G"] < 4096 else ""),
                     "graphs": wb["G"], "n": ub.n, "edges_directed": ub.nnz,
                     "value": job_rate(ub.nnz, args.steps, world, bms / 1e3), "unit": UNIT,
                     "ms_per_step": bms / args.steps, "schedule": "default, concurrent bins",
                     "pass_ms": [round(q["move_ms"] + q["aggregate_ms"], 3) for q in bst["per_pass"]]}
        del dub

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = SAMPLES[args.workload]
        gs, snnz = sample_graphs(sample)
        dt, cores = oracle_steps(gs, 1, 0)
        cpu = {"value": snnz / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{sample['desc']}: {snnz} entries, one whole run per graph, {dt:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": w["desc"], "n": g.n, "edges_directed": g.nnz, "mode": "plain",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2 (CSR {(g.offsets.nbytes + g.cols.nbytes) / 1e9:.2f} GB), no flush",
                       **summary},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu, "clocks": clk,
            "learned_skip": learned, "asynchronous": asynchronous, "leiden": leiden, "sequential": sequential,
            "batch": batch_leg,
            "autotune": tune,
            "phases_ms": {"move": st["move_ms"], "aggregate": st["aggregate_ms"], "other": st["other_ms"]},
            "kernels_ms_warmup": {k: round(v["ms"], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:8]},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
