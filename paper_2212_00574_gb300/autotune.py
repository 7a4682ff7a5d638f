"""Autotuner of the AUTO path choice between the bitset sweep and the
tensor-core form.

It times both paths to their fixpoint on seeded k-partite graphs over a grid
of n, k and edge density, and turns the times into the table that
``kz_api.cu`` compiles in (``kTensorTable``): a cell is 1 where the tensor
form was faster.  A graph falls into the cell of the nearest measured point:
n below 3072, 6144, 12288 or larger; k below 18 or not; density below
0.075, 0.15, 0.25, 0.375 or not.

``autotune_grid.json`` next to this file holds the measurements the
committed table was read from; ``tests/test_autotune.py`` checks that the
two agree.

    python -m paper_2212_00574_gb300.autotune --n 2048,4096,8192,16384 \\
        --p 0.05,0.1,0.2,0.3,0.45 --k 12,24 [--out grid.json]

measures on the current GPU and prints the table as C.  With ``--batch`` it
instead times the fused batch (KZ_BATCH_FUSED) on the 1024-graph workload for
a grid of its cost-model settings (group spread, items per warp, largest
group; kz_set_batch_tuning) and prints the fastest as the constants that
``kz_batch.cu`` compiles in; ``autotune_batch.json`` holds the measurements
the committed constants were read from.
"""
from __future__ import annotations

import argparse
import json
import os

N_EDGES = (3072, 6144, 12288)          # n bins: below each edge, then the rest
K_EDGE = 18                            # k bins: below, then the rest
D_EDGES = (0.075, 0.15, 0.25, 0.375)   # density bins: below each edge, then the rest

GRID_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_grid.json")


def _bin(x, edges):
    for i, e in enumerate(edges):
        if x < e:
            return i
    return len(edges)


def cell(n: int, k: int, density: float) -> tuple[int, int, int]:
    """The table cell of a graph: (n bin, k bin, density bin)."""
    return _bin(n, N_EDGES), int(k >= K_EDGE), _bin(density, D_EDGES)


def table_from(records) -> list:
    """Table [n bin][k bin][density bin] -> 1 where the tensor form was faster
    over the cell's measured graphs (their times summed per path; 0 where
    nothing was measured)."""
    nbins = (len(N_EDGES) + 1, 2, len(D_EDGES) + 1)
    sums = {}
    for r in records:
        c = cell(int(r["n"]), int(r["k"]), float(r["p"]))
        b, tt = sums.get(c, (0.0, 0.0))
        sums[c] = (b + float(r["bitset_us"]), tt + float(r["tensor_us"]))
    t = [[[0] * nbins[2] for _ in range(nbins[1])] for _ in range(nbins[0])]
    for (nb, kb, db), (b, tt) in sums.items():
        t[nb][kb][db] = int(tt < b)
    return t


def render_c(t) -> str:
    """The table as the C initializer of kTensorTable."""
    rows = []
    for nb, per_k in enumerate(t):
        inner = ", ".join("{" + ", ".join(str(v) for v in per_k[kb]) + "}" for kb in range(2))
        rows.append("    {" + inner + "},")
    return "constexpr int kTensorTable[%d][2][%d] = {\n%s\n};" % (len(t), len(D_EDGES) + 1, "\n".join(rows))


def measure(ns, ps, ks, seed: int = 11, runs: int = 5, warm: int = 2):
    """Time both paths to their fixpoint (CUDA events around kz_kernelize,
    L2 flushed between runs, median after the warm-up runs)."""
    import numpy as np
    import torch

    import paper_2212_00574_gb300 as kz
    from paper_2212_00574_gb300 import synth

    dev = torch.device("cuda", 0)
    kz.use_torch_allocator()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    records = []
    for n in ns:
        for k in ks:
            for p in ps:
                g = synth.kpartite(n, k, p, seed=seed, planted=True)
                h = kz.kz_load_graph_dense(g.n, g.k, g.colour, g.get_bits(), stream=stream)
                rec = dict(n=n, k=k, p=p)
                for path in ("bitset", "tensor"):
                    opts = kz.kz_default_options(path=path)
                    times = []
                    for i in range(runs):
                        kz.kz_reset(h, stream)
                        flush.fill_(i)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        kz.kz_kernelize(h, opts, stream)
                        e1.record(stream)
                        torch.cuda.synchronize()
                        times.append(e0.elapsed_time(e1))
                    st = kz.kz_fetch_stats(h)
                    rec[path + "_us"] = round(1e3 * float(np.median(times[warm:])), 1)
                    rec["passes"] = st["passes"]
                kz.kz_free_graph(h)
                records.append(rec)
                print(json.dumps(rec), flush=True)
    return records


# ---------------------------------------------------------------------------
# the fused batch's cost model (kz_set_batch_tuning)
# ---------------------------------------------------------------------------

BATCH_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_batch.json")


def best_batch_tuning(records) -> tuple:
    """(group_spread, items_per_warp, max_group) of the fastest measured
    fused batch."""
    r = min(records, key=lambda r: float(r["fused_ms"]))
    return float(r["group_spread"]), int(r["items_per_warp"]), int(r["max_group"])


def render_batch_c(best) -> str:
    spread, ipw, mg = best
    return ("constexpr int kMaxGroup = %d;\nconstexpr double kGroupSpread = %s;\nconstexpr int kItemsPerWarp = %d;"
            % (mg, repr(float(spread)), ipw))


def measure_batch(spreads, items, groups, count: int = 1024, runs: int = 7, warm: int = 2):
    """Time the fused batch (one kz_kernelize_batch call, KZ_BATCH_FUSED) on
    the 1024-graph workload's recipe for each cost-model setting; the
    concurrent mode is timed once beside it for reference."""
    import numpy as np
    import torch

    import paper_2212_00574_gb300 as kz
    from paper_2212_00574_gb300 import synth

    dev = torch.device("cuda", 0)
    kz.use_torch_allocator()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    specs = synth.batch_specs(count, synth.workload_seed("c4"))
    hs = []
    for (n, k, p, pl, seed) in specs:
        g = synth.kpartite(n, k, p, seed, planted=pl)
        hs.append(kz.kz_load_graph_dense(g.n, g.k, g.colour, g.get_bits(), stream=stream))

    def time_mode(mode):
        opts = kz.kz_default_options(batch=mode)
        times = []
        for i in range(runs):
            for h in hs:
                kz.kz_reset(h, stream)
            flush.fill_(i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            kz.kz_kernelize_batch(hs, opts, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return round(float(np.median(times[warm:])), 3)

    records = []
    concurrent = time_mode("concurrent")
    for mg in groups:
        for s in spreads:
            for ipw in items:
                kz.kz_set_batch_tuning(s, ipw, mg)
                rec = dict(group_spread=s, items_per_warp=ipw, max_group=mg, fused_ms=time_mode("fused"),
                           concurrent_ms=concurrent)
                records.append(rec)
                print(json.dumps(rec), flush=True)
    kz.kz_set_batch_tuning(0, 0, 0)
    for h in hs:
        kz.kz_free_graph(h)
    return records


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", default="2048,4096,8192,16384")
    ap.add_argument("--p", default="0.05,0.1,0.2,0.3,0.45")
    ap.add_argument("--k", default="12,24")
    ap.add_argument("--batch", action="store_true",
                    help="tune the fused batch's cost model on the 1024-graph workload instead")
    ap.add_argument("--spread", default="8,16,32,64,128")
    ap.add_argument("--items", default="1,2,4,8")
    ap.add_argument("--groups", default="64,152,456")
    ap.add_argument("--out", default=None, help="write the measurements as JSON")
    args = ap.parse_args(argv)
    if args.batch:
        records = measure_batch([float(x) for x in args.spread.split(",")], [int(x) for x in args.items.split(",")],
                                [int(x) for x in args.groups.split(",")])
        if args.out:
            with open(args.out, "w") as f:
                json.dump({"records": records}, f, indent=1)
        print(render_batch_c(best_batch_tuning(records)))
        return 0
    records = measure([int(x) for x in args.n.split(",")], [float(x) for x in args.p.split(",")],
                      [int(x) for x in args.k.split(",")])
    if args.out:
        with open(args.out, "w") as f:
            json.dump({"records": records}, f, indent=1)
    print(render_c(table_from(records)))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
