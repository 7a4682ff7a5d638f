"""Benchmark of the colour-index kernelization hot path.

One step = kernelize one graph to its fixpoint (every pass of the vertex and
edge rules until nothing is deleted) from its loaded state.  The default
workload is the largest single-GPU one: the dense random k-partite graph
n=32768, k=24, p=0.85 with a planted 24-clique (437M edges).  The default run
also measures, in the same process and on the same GPU, the two comparisons
the metric asks for:

* learned vs plain: the learned schedule (an MLP trained first, by the
  library's own kernels, on plain-method traces of other graphs) against
  plain Jacobi sweeps, on the same graph and on a cascading graph of the same
  size;
* batched vs plain: the 1024-graph batch kernelized by one kz_kernelize_batch
  call (concurrent streams, or one fused persistent launch) against the plain
  per-graph loop (one kz_kernelize after another).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank kernelizes its own
replica of the workload (independent problems: no data-path collective); the
value is the sum over ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_DESC = {
    "c1": "random k-partite n=300 k=10 p=0.7, planted 10-clique (uint64-bit dense input)",
    "c2": "random k-partite n=4096 k=20 p=0.92, planted 20-clique (dense 0/1 input)",
    "c5": "random k-partite n=32768 k=24 p=0.85, planted 24-clique (dense 0/1 input)",
    "c3": "Chung-Lu n=200000 k=12, Zipf(1.2) class sizes, power-law degrees (exponent 2.3, mean 60), "
          "~6M edges, 5 planted 12-cliques (edge-list input)",
    "c5c": "random k-partite n=32768 k=24 p=0.12, planted 24-clique: the C5 size where the tensor form wins "
           "(dense 0/1 input)",
    "c5s": "random k-partite n=32768 k=24 p=0.07, planted 24-clique: the C5 size in the cascade regime "
           "(dense 0/1 input)",
    "c4": "batch of 1024 random k-partite graphs, n log-uniform [64,4096], k U{6..32}, p U[0.3,0.95], "
          "planted k-clique on even indices, one kz_kernelize_batch call",
}
METRIC = "time-to-fixpoint per graph & edge-rule tests/s, learned/batched vs plain"
UNIT = "edge tests/s"
L2_FLUSH_BYTES = 256 << 20
PROFILES = os.path.join(ROOT, "profiles")
# the source files each profiled kernel is compiled from: a traffic record in
# profiles/ counts only while their hash is the one it was captured with
KERNEL_SOURCES = {
    "bitset_persistent_kernel": ["kz_bitset.cu", "kz_rules.cuh", "kz_sweep.cuh", "kz_state.cuh"],
    "bitset_sweep_kernel": ["kz_bitset.cu", "kz_rules.cuh", "kz_sweep.cuh", "kz_state.cuh"],
    "tensor_edge_kernel": ["kz_tensor.cu", "kz_state.cuh"],
    "sparse_triangle_kernel": ["kz_sparse.cu", "kz_state.cuh"],
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOAD_DESC), default="c5")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU work budget of the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the learned-vs-plain and batched-vs-plain comparisons of the default run")
    ap.add_argument("--compare-steps", type=int, default=10, help="timed steps of each comparison arm")
    ap.add_argument("--clique-k", type=int, default=0,
                    help="clique size q sought (0: q = k); q < k lowers both rule thresholds")
    ap.add_argument("--tensor-precision", choices=["fp8", "bf16"], default="fp8",
                    help="tensor path operands: E4M3 (kind::f8f6f4) or BF16 (kind::f16)")
    ap.add_argument("--dominance", choices=["none", "vertex", "edge"], default="none",
                    help="rounds of vertex (Definition 4.3.1) or edge (Definitions 4.3.2-4.3.3) dominance after "
                         "the colour-index fixpoint")
    ap.add_argument("--max-clique", action="store_true",
                    help="time the maximum-clique driver (kernelize for q = k, k-1, ... and search each kernel)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload (n x scale; for small profiler captures, not for bench lines)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--path", choices=["auto", "bitset", "small", "sparse", "tensor"], default="auto")
    ap.add_argument("--schedule", choices=["plain", "support", "learned"], default="plain",
                    help="plain Jacobi sweeps; the same sweeps with incremental support counts (CSR state); "
                         "or the learned schedule alone, timed against plain")
    ap.add_argument("--plane0", choices=["auto", "full", "half", "two"], default="auto",
                    help="first test of the bitset sweep kernels (full words or half words per class)")
    ap.add_argument("--loop", choices=["device", "graph", "host"], default="device",
                    help="pass loop: device = one cooperative persistent launch, graph = CUDA-graph while "
                         "node, host = one launch per pass from the host")
    return ap.parse_args()


def default_headline(args) -> bool:
    """The default run: the headline workload with no option changed, so the
    comparisons belong on its line."""
    return (args.workload == "c5" and args.schedule == "plain" and args.path == "auto" and args.scale == 1.0
            and args.clique_k == 0 and args.dominance == "none" and args.plane0 == "auto" and args.loop == "device"
            and args.tensor_precision == "fp8" and not args.no_compare)


# ---------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def reduce_max(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() and pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() and pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"kz_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# DRAM traffic records of profiles/
# ---------------------------------------------------------------------------

def sources_sha256(files) -> str:
    """sha256 over the named kernel source files (csrc/), in order."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2212_00574_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_records() -> list:
    """The ```traffic-record blocks of the ncu summaries in profiles/: one
    kernel on one workload, its DRAM bytes (read + write) per launch, and the
    hash of the sources it was compiled from when captured."""
    out = []
    for path in sorted(glob.glob(os.path.join(PROFILES, "*.md"))):
        with open(path) as f:
            lines = f.read().splitlines()
        i = 0
        while i < len(lines):
            if lines[i].strip() == "```traffic-record":
                rec = {"file": os.path.relpath(path, ROOT)}
                i += 1
                while i < len(lines) and lines[i].strip() != "```":
                    if ":" in lines[i]:
                        key, val = lines[i].split(":", 1)
                        rec[key.strip()] = val.strip()
                    i += 1
                out.append(rec)
            i += 1
    return out


def measured_traffic(workload: str, kernel: str):
    """DRAM bytes per launch of `kernel` on `workload` from a committed ncu
    summary, or None when there is none for the kernel as it is now."""
    files = KERNEL_SOURCES.get(kernel)
    if not files:
        return None, None
    now = sources_sha256(files)
    for rec in traffic_records():
        if rec.get("workload") == workload and rec.get("kernel") == kernel and rec.get("sources_sha256") == now:
            return float(rec["dram_bytes_per_launch"]), rec["file"]
    return None, None


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def wdesc(args):
    d = WORKLOAD_DESC[args.workload]
    return d if args.scale == 1.0 else f"{d}, scaled to n x {args.scale:g} (profiling case)"


def make_workload(name, scale=1.0):
    from paper_2212_00574_gb300 import synth
    return synth.workload(name, scale)


def workload_seed(name: str) -> int:
    from paper_2212_00574_gb300 import synth
    return synth.workload_seed(name)


def cpu_baseline(g, budget_s: float, session=None) -> dict:
    """The oracle as it stands, single-threaded, on a bounded sample: the
    edge-rule colour index of uniformly sampled edges of the same graph
    (adjacency lists built once beforehand, as the GPU path loads once)."""
    import oracle
    edges = g.get_edges()
    sess = session or oracle.Session(g.colour, edges, g.k)
    rng = np.random.default_rng(7)
    pilot = rng.choice(len(edges), size=min(len(edges), 300), replace=False).astype(np.int64)
    t0 = time.perf_counter()
    sess.edge_index(pilot)
    per_edge = max((time.perf_counter() - t0) / max(len(pilot), 1), 1e-8)
    size = int(min(len(edges), max(len(pilot), budget_s / per_edge)))
    sample = rng.choice(len(edges), size=size, replace=False).astype(np.int64)
    t0 = time.perf_counter()
    sess.edge_index(sample)
    dt = time.perf_counter() - t0
    if session is None:
        sess.close()
    return {"value": size / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "seconds": round(dt, 3), "edges": size,
            "sample": f"edge-rule colour index of {size} uniformly sampled edges of the same graph "
                      f"(single-threaded C oracle; adjacency lists built once, untimed)"}


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, world, rank, pg):
    if rank != 0:
        return 0
    import oracle
    g = make_workload(args.workload, args.scale)
    sess = oracle.Session(g.colour, g.get_edges(), g.k)
    # every step a bounded sample, so that the whole run ends within minutes
    budget = min(max(60.0 / max(args.steps + args.warmup, 1), 0.01), 2.0)
    per_step = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(g, budget, session=sess)
        if i >= args.warmup:
            per_step.append(cb)
    sess.close()
    value = statistics.median([c["value"] for c in per_step])
    ms = 1e3 * statistics.median([c["seconds"] for c in per_step])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": wdesc(args), "n": g.n, "k": g.k, "m": g.m, "seed": workload_seed(args.workload),
                   "l2": "n/a (CPU)", "parallelism": "single (rank 0 only)"},
        "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": UNIT,
                         "sample": per_step[0]["sample"] + " per step"},
        "extrapolated_ms_per_full_pass": 1e3 * g.m / value,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def timed_steps(kz, torch, handles, run, stream, flush, steps, warmup, local, pg=None):
    """W untimed steps, then K steps timed with CUDA events on the launching
    stream around `run()` only; every step first restores the loaded graphs
    (kz_reset) and flushes L2, outside the events."""
    dev = torch.device("cuda", local)

    def step(i, ev0=None, ev1=None):
        for h in handles:
            kz.kz_reset(h, stream)
        flush.fill_(i & 0xFF)
        if ev0 is not None:
            ev0.record(stream)
        run()
        if ev1 is not None:
            ev1.record(stream)

    for i in range(warmup):
        step(i)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize(dev)
    clocks.start()
    t0 = time.perf_counter()
    for i in range(steps):
        step(i, *evs[i])
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    barrier(pg)
    per_ms = [a.elapsed_time(b) for a, b in evs]
    return {"per_ms": per_ms, "ms": sum(per_ms) / len(per_ms), "median_ms": statistics.median(per_ms),
            "wall_s": wall, "clocks": clk}


def roofline_of(kz, torch, g, st, step_ms, workload, args, dev, stream):
    """Roofline of the dominant kernel of one plain run."""
    passes = max(st["passes"], 1)
    launch_s = step_ms / passes / 1e3
    kernel = {1: "bitset_persistent_kernel", 2: "cta_fixpoint_kernel", 3: "sparse_triangle_kernel",
              4: "tensor_edge_kernel"}.get(st["path"], "?")
    if kernel == "bitset_persistent_kernel" and args.loop != "device":
        kernel = "bitset_sweep_kernel"
    traffic, traffic_src = measured_traffic(workload, kernel)
    if kernel == "tensor_edge_kernel":
        # the tensor form's work is fixed by the shapes: per upper-triangle
        # 128 x 128 tile and per K-step (32 vertices of one class), one
        # M = N = 128, K = 32 MMA (2 * 128 * 128 * 32 flops); peak = the
        # measured bf16 dense peak x 2 (the nominal fp8 : bf16 ratio)
        k = g.k
        sizes = np.bincount(np.asarray(g.colour), minlength=k)
        ksteps = int(sum((int(c) + 31) // 32 for c in sizes))
        t_side = (g.n + 127) // 128
        flops = 2.0 * 128 * 128 * 32 * ksteps * t_side * (t_side + 1) / 2
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        mult = 1.0 if args.tensor_precision == "bf16" else 2.0
        peak = mult * peaks["bf16_tflops_sustained"] * 1e12
        return {"bound": "tensor", "achieved": flops / launch_s / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": flops / launch_s / peak, "traffic": traffic,
                "traffic_source": traffic_src, "kernel": kernel, "flops_per_launch": flops,
                "note": "flops = 2*128*128*32 per (upper-triangle tile, K-step); peak = measured bf16 sustained "
                        f"x {mult:g} (nominal fp8:bf16), of measured; launch time = CUDA events around "
                        "kz_kernelize / passes (includes the expand and commit kernels of each pass)"}
    # The binding operation of the bitset sweep is the word AND of one class
    # word of u's row with v's (a LOP3 on the 64-lane integer logic pipe); the
    # zero test runs on the separate min pipe.  Algorithmic ANDs per launch =
    # live edges tested x (k-2) needed classes (one plane-0 word each on a
    # dense graph).
    alg_ops = st["edge_tests"] / passes * max(g.k - 2, 0)
    probe_ops, _ = kz.kz_probe_int_throughput(0, stream)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 64 * 2.070e9
    return {"bound": "alu", "achieved": alg_ops / launch_s / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
            "frac": alg_ops / launch_s / peak, "traffic": traffic, "traffic_source": traffic_src,
            "kernel": kernel, "probe_lop3_tops": probe_ops / 1e12, "ops_per_launch": alg_ops,
            "note": "ops = live edges tested x (k-2) class-word ANDs; peak = SMs x 64 logic lanes x 2070 MHz "
                    "(derived from unit counts and the maximum clock; the LOP3 probe measures it); launch "
                    "time = CUDA events around kz_kernelize / passes (includes the run-start kernel); traffic "
                    "= DRAM bytes read + written per launch from the committed ncu summary named in "
                    "traffic_source (null when none matches the kernel's current sources)"}


# multiply-adds per scored edge of the 16 -> 64 -> 64 -> 1 network, x 2 flops
MLP_FLOPS_PER_EDGE = 2 * (16 * 64 + 64 * 64 + 64)


def mlp_roofline(kz, torch, model, stream, rows=1 << 22, reps=10):
    """The network's forward kernel (bf16 mma.sync, fp32 accumulation; the
    scoring kernel runs the same tile code after computing the features) on
    `rows` feature rows, against the measured dense bf16 peak."""
    X = torch.randn(rows, 16, device="cuda", dtype=torch.float32)
    out = torch.empty(rows, device="cuda", dtype=torch.float32)
    for _ in range(3):
        kz.kz_mlp_forward(model, X.data_ptr(), rows, out.data_ptr(), stream)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        kz.kz_mlp_forward(model, X.data_ptr(), rows, out.data_ptr(), stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    s = statistics.median(times)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    peak = peaks["bf16_tflops"] * 1e12
    flops = MLP_FLOPS_PER_EDGE * rows
    return {"bound": "tensor", "kernel": "mlp_forward_kernel", "rows": rows, "flops_per_edge": MLP_FLOPS_PER_EDGE,
            "achieved": flops / s / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": flops / s / peak,
            "us": 1e6 * s, "bytes_per_edge": 16 * 4 + 4, "hbm_gbs": (16 * 4 + 4) * rows / s / 1e9,
            "note": "peak = measured dense bf16 burst (cuBLAS), of measured; the kernel runs on the legacy "
                    "warp-level mma.sync path"}


def learned_comparison(kz, torch, graphs, stream, flush, local, args, pg, rank):
    """Train the edge-scoring network (plain-method traces of cascading graphs
    with other seeds; the library's forward/backward/Adam kernels), then time
    the learned schedule against plain sweeps on each given graph, checking
    that the two kernels are bit-identical."""
    from paper_2212_00574_gb300 import learned, synth
    t0 = time.perf_counter()
    X, y = learned.collect(learned.cascade_specs(24, synth.SEED_BASE + 900 + rank), per_sweep_cap=3000)
    model, losses = learned.train(X, y, steps=300, batch=4096, lr=3e-3)
    train_s = time.perf_counter() - t0
    mlp = mlp_roofline(kz, torch, model, stream)
    out = {"mlp_roofline": mlp,
           "training": {"records": int(len(y)), "positive_share": float(np.mean(y)), "loss_first": losses[0],
                        "loss_last": losses[-1], "seconds": round(train_s, 2),
                        "graphs": "24 cascading k-partite graphs (n log-uniform 256..32768, k 8..32, p = sqrt(mu k / n) with mu 3..9), other seeds"}}
    try:
        arms = (("plain", "plain", None), ("learned", "learned", 0.5), ("frontier", "learned", 0.0),
                ("support", "support", None))
        for name, g, h in graphs:
            res = {}
            for label, sched, thr in arms:
                if thr is not None:
                    kz.kz_attach_model(h, model, thr)
                opts = kz.kz_default_options(schedule=sched)
                t = timed_steps(kz, torch, [h], lambda: kz.kz_kernelize(h, opts, stream), stream, flush,
                                args.compare_steps, 2, local, pg)
                st = kz.kz_fetch_stats(h)
                alive, bits, _ = kz.kz_fetch_kernel_dense(h, g.n)
                res[label] = dict(ms=t["median_ms"], st=st, alive=alive, bits=bits, clocks=t["clocks"])
            same = all(np.array_equal(res["plain"]["alive"], res[a]["alive"])
                       and np.array_equal(res["plain"]["bits"], res[a]["bits"]) for a, _, _ in arms)
            p, lr = res["plain"], res["learned"]
            labels = [a for a, _, _ in arms]
            out[name] = {"time_to_fixpoint_ms": {a: res[a]["ms"] for a in labels},
                         "speedup": p["ms"] / lr["ms"],
                         "speedup_frontier_only": p["ms"] / res["frontier"]["ms"],
                         "speedup_support": p["ms"] / res["support"]["ms"],
                         "plain_path": {v: k for k, v in kz.PATHS.items()}.get(p["st"]["path"]),
                         "sweeps": {a: res[a]["st"]["sweeps"] for a in labels},
                         "passes": {a: res[a]["st"]["passes"] for a in labels},
                         "edge_tests": {a: res[a]["st"]["edge_tests"] for a in labels},
                         "kernel_edges": p["st"]["m_live"], "bit_identical": same,
                         "sm_mhz": lr["clocks"].get("sm_mhz"), "reasons": lr["clocks"].get("reasons")}
    finally:
        kz.kz_model_free(model)
    return out


def batch_comparison(kz, torch, stream, flush, local, args, pg):
    """The 1024-graph batch: the plain per-graph loop (kz_kernelize on each
    graph in turn) against one kz_kernelize_batch call, concurrent and
    fused; every mode must leave every graph with the same kernel."""
    from paper_2212_00574_gb300 import synth
    specs = synth.batch_specs(1024, synth.workload_seed("c4"))
    graphs = [synth.kpartite(n, k, p, seed, planted=pl) for (n, k, p, pl, seed) in specs]
    handles = [kz.kz_load_graph_dense(g.n, g.k, g.colour, g.get_bits(), stream=stream) for g in graphs]
    plain = kz.kz_default_options()
    modes = {
        "plain_loop": lambda: [kz.kz_kernelize(h, plain, stream) for h in handles],
        "batch_concurrent": lambda: kz.kz_kernelize_batch(handles, kz.kz_default_options(batch="concurrent"),
                                                          stream),
        "batch_fused": lambda: kz.kz_kernelize_batch(handles, kz.kz_default_options(batch="fused"), stream),
    }
    res, ref = {}, None
    try:
        for label, run in modes.items():
            t = timed_steps(kz, torch, handles, run, stream, flush, args.compare_steps, 2, local, pg)
            sts = [kz.kz_fetch_stats(h) for h in handles]
            sig = [(s["n_live"], s["m_live"], s["sweeps"]) for s in sts]
            if ref is None:
                ref = sig
            res[label] = dict(ms=t["median_ms"], tests=sum(s["edge_tests"] for s in sts), same=(sig == ref),
                              sweeps_max=max(s["sweeps"] for s in sts), clocks=t["clocks"])
    finally:
        for h in handles:
            kz.kz_free_graph(h)
    base = res["plain_loop"]["ms"]
    return {"graphs": len(graphs), "m_total": int(sum(g.m for g in graphs)),
            "time_to_fixpoint_ms_per_batch": {k: v["ms"] for k, v in res.items()},
            "time_to_fixpoint_us_per_graph": {k: 1e3 * v["ms"] / len(graphs) for k, v in res.items()},
            "speedup_vs_plain_loop": {k: base / v["ms"] for k, v in res.items() if k != "plain_loop"},
            "edge_tests": res["plain_loop"]["tests"], "sweeps_max": res["plain_loop"]["sweeps_max"],
            "same_kernels": all(v["same"] for v in res.values()),
            "sm_mhz": res["batch_concurrent"]["clocks"].get("sm_mhz"),
            "reasons": sorted(set(sum((v["clocks"].get("reasons") or [] for v in res.values()), [])))}


def run_ours(args, world, rank, local, pg):
    import torch

    import paper_2212_00574_gb300 as kz

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kz.use_torch_allocator()
    g = make_workload(args.workload, args.scale)
    stream = torch.cuda.current_stream(dev)
    dense = args.workload != "c3"
    pin_col = torch.from_numpy(g.colour).pin_memory()
    h_col = pin_col.numpy()
    if dense:
        bits = g.get_bits()
        # pinned host copies of the inputs (for the end-to-end measurement)
        pin_bits = torch.from_numpy(bits.view(np.int64)).pin_memory()
        h_bits = pin_bits.numpy().view(np.uint64)
        h = kz.kz_load_graph_dense(g.n, g.k, h_col, h_bits, stream=stream)
    else:
        pin_edges = torch.from_numpy(g.get_edges()).pin_memory()
        h_edges = pin_edges.numpy()
        h = kz.kz_load_graph(g.n, g.k, h_col, h_edges, stream=stream)
    opts = kz.kz_default_options(path=args.path, use_graph={"device": 1, "graph": 2, "host": 0}[args.loop],
                                 plane0={"auto": 0, "full": 1, "half": 2, "two": 3}[args.plane0],
                                 schedule=args.schedule, clique_k=args.clique_k,
                                 dominance={"none": 0, "vertex": 1, "edge": 2}[args.dominance],
                                 tensor_precision=1 if args.tensor_precision == "bf16" else 0)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    t = timed_steps(kz, torch, [h], lambda: kz.kz_kernelize(h, opts, stream), stream, flush, args.steps,
                    args.warmup, local, pg)
    st = kz.kz_fetch_stats(h)
    tests_per_step, passes = st["edge_tests"], st["passes"]
    dev_ms = sum(t["per_ms"])
    slowest_s = reduce_max(pg, dev_ms / 1e3)
    value = reduce_sum(pg, float(tests_per_step) * args.steps) / slowest_s
    ms_per_step = dev_ms / args.steps
    roofline = roofline_of(kz, torch, g, st, ms_per_step, args.workload if args.scale == 1.0 else None, args,
                           dev, stream)

    # end to end through the C ABI: host buffers in, host buffers out, every
    # copy inside the timed region
    e2e = None
    if args.e2e_steps > 0 and not dense:
        times = []
        for i in range(args.e2e_steps + 1):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            hh = kz.kz_load_graph(g.n, g.k, h_col, h_edges, stream=stream)
            kz.kz_kernelize(hh, opts, stream)
            alive_o, kept, _ = kz.kz_fetch_kernel(hh, g.n)
            kz.kz_free_graph(hh)
            dt = time.perf_counter() - t0
            if i >= 1:
                times.append(dt)
        e2e_s = statistics.median(times)
        e2e = {"value": tests_per_step * world / reduce_max(pg, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(h_edges.nbytes + h_col.nbytes),
               "d2h_bytes_per_step": int(alive_o.nbytes + kept.nbytes), "ms_per_step": 1e3 * e2e_s,
               "calls": "kz_load_graph + kz_kernelize + kz_fetch_kernel + kz_free_graph"}
    if args.e2e_steps > 0 and dense:
        out_bits = torch.empty((g.n, bits.shape[1]), dtype=torch.int64).pin_memory().numpy().view(np.uint64)
        out_alive = torch.empty(g.n, dtype=torch.uint8).pin_memory().numpy()
        # the device-resident run's kernel, to check the end-to-end result against
        kz.kz_fetch_kernel_dense(h, g.n, out_bits=out_bits, out_alive=out_alive)
        ref_bits, ref_alive = out_bits.copy(), out_alive.copy()
        times = []
        for i in range(args.e2e_steps + 2):
            flush.fill_(i & 0xFF)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            hh = kz.kz_load_graph_dense(g.n, g.k, h_col, h_bits, stream=stream)
            kz.kz_kernelize(hh, opts, stream)
            kz.kz_fetch_kernel_dense(hh, g.n, out_bits=out_bits, out_alive=out_alive)
            kz.kz_free_graph(hh)
            dt = time.perf_counter() - t0
            if i >= 2:
                times.append(dt)
        assert np.array_equal(out_bits, ref_bits) and np.array_equal(out_alive, ref_alive)
        e2e_s = statistics.median(times)
        e2e = {"value": tests_per_step * world / reduce_max(pg, e2e_s),
               "unit": UNIT, "h2d_bytes_per_step": int(h_bits.nbytes + h_col.nbytes),
               "d2h_bytes_per_step": int(out_bits.nbytes + out_alive.nbytes),
               "ms_per_step": 1e3 * e2e_s,
               "calls": "kz_load_graph_dense + kz_kernelize + kz_fetch_kernel_dense + kz_free_graph"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g, args.cpu_seconds)

    comparisons = None
    if default_headline(args):
        gs = make_workload("c5s")
        hs = kz.kz_load_graph_dense(gs.n, gs.k, gs.colour, gs.get_bits(), stream=stream)
        try:
            comparisons = {"learned_vs_plain": learned_comparison(kz, torch, [("c5", g, h), ("c5s", gs, hs)],
                                                                  stream, flush, local, args, pg, rank)}
        finally:
            kz.kz_free_graph(hs)
        comparisons["batched_vs_plain"] = batch_comparison(kz, torch, stream, flush, local, args, pg)
        comparisons["workloads"] = {"c5": WORKLOAD_DESC["c5"], "c5s": WORKLOAD_DESC["c5s"],
                                    "c4": WORKLOAD_DESC["c4"]}
        comparisons["timing"] = (f"median of {args.compare_steps} steps after 2 warm-up steps, CUDA events around "
                                 "the kernelize call(s) only, kz_reset and an L2 flush between steps")
    kz.kz_free_graph(h)

    # our kernels inside one timed step: the reset kernel runs outside the
    # events; inside, the run-start kernel and one persistent launch (bitset),
    # or per pass the expand, tensor and commit kernels (tensor)
    per_step = {1: 2, 2: 2, 3: 1 + 4 * passes, 4: 1 + 3 * passes}.get(st["path"], 1 + passes)
    if rank == 0:
        tt = sorted(t["per_ms"])
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wdesc(args), "n": g.n, "k": g.k, "m": g.m,
                       "seed": workload_seed(args.workload),
                       "path": {v: k for k, v in kz.PATHS.items()}.get(st["path"], str(st["path"])),
                       "pass_loop": {"device": "one cooperative persistent launch", "graph": "CUDA-graph while node",
                                     "host": "host-driven"}[args.loop],
                       "passes": passes, "sweeps": st["sweeps"], "schedule": args.schedule,
                       "clique_k": st["clique_k"], "dominance_rounds": st["dominance_rounds"],
                       "dominated": st["dominated"],
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write); per-step CUDA events "
                             "around kz_kernelize only",
                       "parallelism": "replicas" if world > 1 else "single"},
            "time_to_fixpoint_us": {"median": 1e3 * tt[len(tt) // 2], "p10": 1e3 * tt[len(tt) // 10],
                                    "p90": 1e3 * tt[(9 * len(tt)) // 10]},
            "wall_s_timed_region": t["wall_s"],
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "comparisons": comparisons,
            "gpu_launches": per_step * args.steps,
            "clocks": t["clocks"],
        }
        print(json.dumps(line), flush=True)
    ok = comparisons is None or (all(v.get("bit_identical", True) for v in comparisons["learned_vs_plain"].values()
                                     if isinstance(v, dict))
                                 and comparisons["batched_vs_plain"]["same_kernels"])
    return 0 if ok else 1


def run_batch(args, world, rank, local, pg):
    """Batched workload alone: one step = the whole 1024-graph batch, in each
    mode (the plain per-graph loop, concurrent, fused)."""
    import torch

    import paper_2212_00574_gb300 as kz

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kz.use_torch_allocator()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    args.compare_steps = args.steps
    b = batch_comparison(kz, torch, stream, flush, local, args, pg)
    ms = b["time_to_fixpoint_ms_per_batch"]["batch_concurrent"]
    slowest = reduce_max(pg, ms * args.steps / 1e3)
    value = reduce_sum(pg, float(b["edge_tests"]) * args.steps) / slowest
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": 2, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC["c4"], "seed": workload_seed("c4"), "graphs": b["graphs"],
                       "m_total": b["m_total"], "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "batched_vs_plain": b,
        }
        print(json.dumps(line), flush=True)
    return 0 if b["same_kernels"] else 1


def run_max_clique(args, world, rank, local, pg):
    """The maximum-clique driver end to end on one graph: for q = k, k-1, ...
    reset, kernelize for clique size q on the GPU, search the kernel (host
    branch and bound), stop at the first q with a clique.  Timed on the wall
    clock (the search runs on the host), after warm-up runs."""
    import torch
    import paper_2212_00574_gb300 as kz
    dev = torch.device("cuda", local)
    kz.use_torch_allocator()
    stream = torch.cuda.current_stream(dev)
    g = make_workload(args.workload, args.scale)
    dense = g.bits is not None
    if dense:
        h = kz.kz_load_graph_dense(g.n, g.k, g.colour, g.get_bits(), stream=stream)
    else:
        h = kz.kz_load_graph(g.n, g.k, g.colour, g.get_edges(), stream=stream)
    opts = kz.kz_default_options(path=args.path)
    times = []
    q = 0
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        q, clique = kz.kz_max_clique(h, g.k, opts, stream=stream)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    st = kz.kz_fetch_stats(h)
    kz.kz_free_graph(h)
    if rank == 0:
        ms = 1e3 * statistics.median(times)
        print(json.dumps({"metric": "maximum-clique time (kernelize for q = k, k-1, ... and search)",
                          "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                          "dtype": "u32", "data": "synthetic",
                          "config": {"workload": wdesc(args), "seed": workload_seed(args.workload), "n": g.n,
                                     "k": g.k, "path": st["path"], "clique_number": q,
                                     "kernel_vertices": st["n_live"], "kernel_edges": st["m_live"],
                                     "parallelism": "single"}}), flush=True)
    return 0


def run_learned(args, world, rank, local, pg):
    """Learned schedule against plain sweeps on the chosen graph alone."""
    import torch

    import paper_2212_00574_gb300 as kz

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kz.use_torch_allocator()
    stream = torch.cuda.current_stream(dev)
    g = make_workload(args.workload, args.scale)
    h = kz.kz_load_graph_dense(g.n, g.k, g.colour, g.get_bits(), stream=stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    args.compare_steps = args.steps
    try:
        cmp = learned_comparison(kz, torch, [(args.workload, g, h)], stream, flush, local, args, pg, rank)
    finally:
        kz.kz_free_graph(h)
    r = cmp[args.workload]
    ms = r["time_to_fixpoint_ms"]["learned"]
    value = reduce_sum(pg, float(r["edge_tests"]["learned"])) / reduce_max(pg, ms / 1e3)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": 2, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": wdesc(args), "seed": workload_seed(args.workload), "n": g.n, "k": g.k,
                       "m": g.m, "schedule": "learned (threshold 0.5)",
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "learned_vs_plain": cmp}), flush=True)
    return 0 if r["bit_identical"] else 1


def main():
    args = parse()
    world, rank, local, pg = dist_init()
    try:
        if args.impl == "reference":
            return run_reference(args, world, rank, pg)
        if args.workload == "c4":
            return run_batch(args, world, rank, local, pg)
        if args.schedule == "learned":
            return run_learned(args, world, rank, local, pg)
        if args.max_clique:
            return run_max_clique(args, world, rank, local, pg)
        return run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
