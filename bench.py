"""Benchmark of the colour-index kernelization hot path.

One step = kernelize one graph to its fixpoint (every pass of the vertex and
edge rules until nothing is deleted) from its loaded state.  The default
workload is the dense random k-partite graph n=4096, k=20, p=0.92 with a
planted 20-clique.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank kernelizes its own
replica of the workload (independent problems: no data-path collective); the
value is the sum over ranks divided by the slowest rank's time.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD_DESC = {
    "c1": "random k-partite n=300 k=10 p=0.7, planted 10-clique (uint64-bit dense input)",
    "c2": "random k-partite n=4096 k=20 p=0.92, planted 20-clique (dense 0/1 input)",
    "c5": "random k-partite n=32768 k=24 p=0.85, planted 24-clique (dense 0/1 input)",
    "c3": "Chung-Lu n=200000 k=12, Zipf(1.2) class sizes, power-law degrees (exponent 2.3, mean 60), "
          "~6M edges, 5 planted 12-cliques (edge-list input)",
    "c5c": "random k-partite n=32768 k=24 p=0.12, planted 24-clique: the C5 size in the cascade regime "
           "(dense 0/1 input)",
    "c4": "batch of 1024 random k-partite graphs, n log-uniform [64,4096], k U{6..32}, p U[0.3,0.95], "
          "planted k-clique on even indices, one kz_kernelize_batch call (graphs spread over streams)",
}
METRIC = "edge-rule tests/s to fixpoint (time-to-fixpoint per graph)"
UNIT = "edge tests/s"
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes read + written by one launch of the dominant kernel, from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum); the summaries with
# the commands are in profiles/.  An entry is removed when its kernel changes.
MEASURED_TRAFFIC = {
    ("c2", "bitset_persistent_kernel"): 2334976,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOAD_DESC), default="c2")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU work budget of the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clique-k", type=int, default=0,
                    help="clique size q sought (0: q = k); q < k lowers both rule thresholds")
    ap.add_argument("--tensor-precision", choices=["fp8", "bf16"], default="fp8",
                    help="tensor path operands: E4M3 (kind::f8f6f4) or BF16 (kind::f16)")
    ap.add_argument("--dominance", action="store_true",
                    help="vertex dominance rounds (Definition 4.3.1) after the colour-index fixpoint")
    ap.add_argument("--max-clique", action="store_true",
                    help="time the maximum-clique driver (kernelize for q = k, k-1, ... and search each kernel)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="shrink the workload (n x scale; for small profiler captures, not for bench lines)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--path", choices=["auto", "bitset", "small", "sparse", "tensor"], default="auto")
    ap.add_argument("--schedule", choices=["plain", "support", "learned"], default="plain",
                    help="plain Jacobi sweeps; the same sweeps with incremental support counts (CSR state); "
                         "or the learned schedule (an MLP trained first, on plain-method traces of "
                         "C4-style cascading graphs, by the library's own kernels), timed against plain")
    ap.add_argument("--plane0", choices=["auto", "full", "half", "two"], default="auto",
                    help="first test of the bitset sweep kernels (full words or half words per class)")
    ap.add_argument("--loop", choices=["device", "graph", "host"], default="device",
                    help="pass loop: device = one cooperative persistent launch, graph = CUDA-graph while "
                         "node, host = one launch per pass from the host")
    return ap.parse_args()


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
# workloads
# ---------------------------------------------------------------------------

def wdesc(args):
    d = WORKLOAD_DESC[args.workload]
    return d if args.scale == 1.0 else f"{d}, scaled to n x {args.scale:g} (profiling case)"


def make_workload(name, scale=1.0):
    from paper_2212_00574_gb300 import synth
    return synth.workload(name, scale)


def cpu_baseline(g, budget_s: float, session=None) -> dict:
    """The oracle as it stands, single-threaded, on a bounded sample: the
    edge-rule colour index of uniformly sampled edges of the same graph
    (adjacency lists built once beforehand, as the GPU path loads once)."""
    import oracle
    edges = g.get_edges()
    sess = session or oracle.Session(g.colour, edges, g.k)
    rng = np.random.default_rng(7)
    pilot = rng.choice(len(edges), size=min(len(edges), 500), replace=False).astype(np.int64)
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
            "seconds": round(dt, 3),
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
    budget = min(max(60.0 / max(args.steps + args.warmup, 1), 0.01), 2.0)
    per_step = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(g, budget, session=sess)
        if i >= args.warmup:
            per_step.append(cb)
    sess.close()
    value = statistics.median([c["value"] for c in per_step])
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * g.m / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": wdesc(args), "n": g.n, "k": g.k, "m": g.m,
                   "l2": "n/a (CPU)", "parallelism": "replicas"},
        "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": UNIT,
                         "sample": per_step[0]["sample"] + " per step; ms_per_step extrapolates "
                                   "the per-edge rate to all edges of one pass"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

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
                                 dominance=1 if args.dominance else 0,
                                 tensor_precision=1 if args.tensor_precision == "bf16" else 0)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(i, ev0=None, ev1=None):
        kz.kz_reset(h, stream)
        flush.fill_(i & 0xFF)
        if ev0 is not None:
            ev0.record(stream)
        kz.kz_kernelize(h, opts, stream)
        if ev1 is not None:
            ev1.record(stream)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    st = kz.kz_fetch_stats(h)
    tests_per_step = st["edge_tests"]
    passes = st["passes"]

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    barrier(pg)
    torch.cuda.synchronize(dev)
    clocks.start()
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        step(i, *evs[i])
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    barrier(pg)
    per_ms = [a.elapsed_time(b) for a, b in evs]
    dev_ms = sum(per_ms)
    st_end = kz.kz_fetch_stats(h)
    assert st_end["edge_tests"] == tests_per_step and st_end["passes"] == passes

    slowest_s = reduce_max(pg, dev_ms / 1e3)
    total_tests = reduce_sum(pg, float(tests_per_step) * args.steps)
    value = total_tests / slowest_s
    ms_per_step = dev_ms / args.steps

    # roofline of the dominant kernel (one sweep-kernel launch per pass).  The
    # binding operation is the word AND of one class word of u's row with v's
    # (a LOP3 on the 64-lane integer logic pipe); the zero test runs on the
    # separate min pipe.  Algorithmic ANDs per launch = live edges tested x
    # (k-2) needed classes (one plane-0 word each on a dense graph).
    k = g.k
    launch_s = (dev_ms / args.steps) / passes / 1e3
    alg_ops = tests_per_step / passes * max(k - 2, 0)
    probe_ops, _ = kz.kz_probe_int_throughput(0, stream)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_derived = sms * 64 * 2.070e9  # 64 32-bit logic lanes per SM (probe-confirmed) x max SM clock
    achieved = alg_ops / launch_s
    kernel = {1: "bitset_persistent_kernel", 2: "cta_fixpoint_kernel", 3: "sparse pass kernels",
              4: "tensor_edge_kernel"}.get(st["path"], "?")
    if kernel == "bitset_persistent_kernel" and args.loop != "device":
        kernel = "bitset_sweep_kernel"
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_derived / 1e12, "unit": "Tops/s",
                "frac": achieved / peak_derived, "traffic": MEASURED_TRAFFIC.get((args.workload, kernel)),
                "kernel": kernel,
                "probe_lop3_tops": probe_ops / 1e12,
                "ops_per_launch": alg_ops,
                "note": "ops = live edges tested x (k-2) class-word ANDs; peak = SMs x 64 logic lanes x "
                        "2070 MHz (derived; the LOP3 probe measures it); launch time = CUDA events around "
                        "kz_kernelize / passes (includes graph-launch overhead); traffic = DRAM bytes read + "
                        "written per launch from one ncu capture of this kernel on this workload (null where "
                        "none was taken for the current kernel)"}

    if kernel == "tensor_edge_kernel":
        # the tensor form's work is fixed by the shapes: per upper-triangle
        # 128 x 128 tile and per K-step (32 vertices of one class), one
        # M = N = 128, K = 32 fp8 MMA (2 * 128 * 128 * 32 flops); peak = the
        # measured bf16 dense peak x 2 (the nominal fp8 : bf16 ratio)
        sizes = np.bincount(np.asarray(g.colour), minlength=k)
        ksteps = int(sum((int(c) + 31) // 32 for c in sizes))
        t_side = (g.n + 127) // 128
        flops = 2.0 * 128 * 128 * 32 * ksteps * t_side * (t_side + 1) / 2
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        fp8_peak = (1.0 if args.tensor_precision == "bf16" else 2.0) * peaks["bf16_tflops"] * 1e12
        roofline = {"bound": "tensor", "achieved": flops / launch_s / 1e12, "peak": fp8_peak / 1e12,
                    "unit": "TFLOP/s", "frac": flops / launch_s / fp8_peak,
                    "traffic": MEASURED_TRAFFIC.get((args.workload, kernel)), "kernel": kernel,
                    "flops_per_launch": flops,
                    "note": "flops = 2*128*128*32 per (upper-triangle tile, K-step); peak = measured bf16 burst "
                            "x 2 (nominal fp8:bf16), of measured; launch time = CUDA events around kz_kernelize "
                            "/ passes (includes the expand and commit kernels of each pass)"}

    # end-to-end through the C ABI: host buffers in, host buffers out
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
    kz.kz_free_graph(h)

    launches_per_step = 2 + passes  # reset-state kernel, run-start kernel, one sweep kernel per pass
    if rank == 0:
        tt = sorted(per_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wdesc(args), "n": g.n, "k": g.k, "m": g.m,
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
            "wall_s_timed_region": t_wall,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    return 0


def run_batch(args, world, rank, local, pg):
    """Batched workload: one step = kz_kernelize_batch over every graph."""
    import torch

    import paper_2212_00574_gb300 as kz
    from paper_2212_00574_gb300 import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kz.use_torch_allocator()
    stream = torch.cuda.current_stream(dev)
    specs = synth.batch_specs(1024, synth.SEED_BASE + 4)
    graphs = [synth.kpartite(n, k, p, seed, planted=pl) for (n, k, p, pl, seed) in specs]
    handles = [kz.kz_load_graph_dense(g.n, g.k, g.colour, g.get_bits(), stream=stream) for g in graphs]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    results = {}
    variants = (("concurrent", "auto", "concurrent"), ("sequential", "auto", "sequential"),
                ("fused_jacobi", "auto", "fused"), ("in_cta_persistent", "small", "fused"))
    for label, path, mode in variants:
        opts = kz.kz_default_options(path=path, batch=mode)

        def step(i, ev0=None, ev1=None):
            for h in handles:
                kz.kz_reset(h, stream)
            flush.fill_(i & 0xFF)
            if ev0 is not None:
                ev0.record(stream)
            kz.kz_kernelize_batch(handles, opts, stream)
            if ev1 is not None:
                ev1.record(stream)

        for i in range(args.warmup):
            step(i)
        torch.cuda.synchronize(dev)
        tests = sum(kz.kz_fetch_stats(h)["edge_tests"] for h in handles)
        sweeps = [kz.kz_fetch_stats(h)["sweeps"] for h in handles]
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        clocks = ClockSampler(local)
        barrier(pg)
        torch.cuda.synchronize(dev)
        clocks.start()
        for i in range(args.steps):
            step(i, *evs[i])
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        barrier(pg)
        per_ms = [a.elapsed_time(b) for a, b in evs]
        results[label] = dict(ms=sum(per_ms) / args.steps, tests=tests, clocks=clk,
                              sweeps_max=max(sweeps), sweeps_total=sum(sweeps))
    for h in handles:
        kz.kz_free_graph(h)
    b = results["concurrent"]
    slowest = reduce_max(pg, b["ms"] * args.steps / 1e3)
    value = reduce_sum(pg, float(b["tests"]) * args.steps) / slowest
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC["c4"], "graphs": len(graphs),
                       "m_total": int(sum(g.m for g in graphs)),
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "time_to_fixpoint_us_per_graph": 1e3 * b["ms"] / len(graphs),
            "other_batch_modes_ms_per_step": {lbl: results[lbl]["ms"] for lbl, _, _ in variants[1:]},
            "sweeps": {"max": b["sweeps_max"], "total": b["sweeps_total"]},
            "clocks": b["clocks"],
        }
        print(json.dumps(line), flush=True)
    return 0


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
                          "config": {"workload": wdesc(args), "n": g.n, "k": g.k, "path": st["path"],
                                     "clique_number": q, "kernel_vertices": st["n_live"],
                                     "kernel_edges": st["m_live"], "parallelism": "single"}}), flush=True)
    return 0


def run_learned(args, world, rank, local, pg):
    """Learned schedule against plain sweeps on one graph: the network is
    trained first (plain-method traces of C4-style cascading graphs with other
    seeds, the library's forward/backward/Adam kernels), then both schedules
    run to the fixpoint from the same loaded graph, the results compared bit
    for bit, and each timed with CUDA events around kz_kernelize."""
    import torch

    import paper_2212_00574_gb300 as kz
    from paper_2212_00574_gb300 import learned, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    kz.use_torch_allocator()
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    X, y = learned.collect(learned.cascade_specs(24, synth.SEED_BASE + 900 + rank), per_sweep_cap=3000)
    model, losses = learned.train(X, y, steps=300, batch=4096, lr=3e-3)
    train_s = time.perf_counter() - t0
    g = make_workload(args.workload, args.scale)
    bits = g.get_bits()
    h = kz.kz_load_graph_dense(g.n, g.k, g.colour, bits, stream=stream)
    kz.kz_attach_model(h, model, 0.5)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    res = {}
    for label, opts in (("plain", kz.kz_default_options(path="bitset")),
                        ("learned", kz.kz_default_options(path="bitset", schedule="learned"))):
        def step(i, ev0=None, ev1=None):
            kz.kz_reset(h, stream)
            flush.fill_(i & 0xFF)
            if ev0 is not None:
                ev0.record(stream)
            kz.kz_kernelize(h, opts, stream)
            if ev1 is not None:
                ev1.record(stream)

        for i in range(args.warmup):
            step(i)
        torch.cuda.synchronize(dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        clocks = ClockSampler(local)
        barrier(pg)
        torch.cuda.synchronize(dev)
        clocks.start()
        for i in range(args.steps):
            step(i, *evs[i])
        torch.cuda.synchronize(dev)
        clk = clocks.stop()
        barrier(pg)
        ms = [a.elapsed_time(b) for a, b in evs]
        st = kz.kz_fetch_stats(h)
        alive, out_bits, _ = kz.kz_fetch_kernel_dense(h, g.n)
        res[label] = dict(ms=sum(ms) / len(ms), tests=st["edge_tests"], sweeps=st["sweeps"], passes=st["passes"],
                          alive=alive.copy(), bits=out_bits.copy(), clocks=clk, dev_s=sum(ms) / 1e3)
    kz.kz_free_graph(h)
    kz.kz_model_free(model)
    same = bool(np.array_equal(res["plain"]["alive"], res["learned"]["alive"])
                and np.array_equal(res["plain"]["bits"], res["learned"]["bits"]))
    lr = res["learned"]
    slowest = reduce_max(pg, lr["dev_s"])
    value = reduce_sum(pg, float(lr["tests"]) * args.steps) / slowest
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": lr["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": wdesc(args), "n": g.n, "k": g.k, "m": g.m,
                       "schedule": "learned (threshold 0.5)", "path": "bitset",
                       "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "time_to_fixpoint_us": {"learned": 1e3 * lr["ms"], "plain": 1e3 * res["plain"]["ms"]},
            "learned_vs_plain": {"speedup_time": res["plain"]["ms"] / lr["ms"],
                                 "tests": {"learned": lr["tests"], "plain": res["plain"]["tests"]},
                                 "sweeps": {"learned": lr["sweeps"], "plain": res["plain"]["sweeps"]},
                                 "bit_identical": same},
            "training": {"records": int(len(y)), "positive_share": float(np.mean(y)), "loss_first": losses[0],
                         "loss_last": losses[-1], "seconds": train_s,
                         "graphs": "24 C4-style cascading graphs (n 128..1500, p 0.15..0.45), other seeds"},
            "clocks": lr["clocks"],
        }
        print(json.dumps(line), flush=True)
    return 0 if same else 1


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
