"""Write the oracle's digests of the full-size workloads.

Runs on the CPU only and calls nothing but the oracle (``oracle/``) and the
seeded input generators (``paper_2212_00574_gb300.synth``, which hold none of
the method's arithmetic).  The GPU parity tests compare the CUDA path's
survivors, sweep counts and per-sweep deletion counts with these digests, so
graphs far too large to re-run through the oracle inside a test are still
checked bit for bit.

Each record holds:

* ``input_sha256``: sha256 of the colour array (int32 little-endian) followed by
  the canonical sorted edge list (int32 pairs).  A test first recomputes it, so
  a generator that draws differently on another machine is reported as such
  rather than as a kernel mismatch.
* ``vlive_sha256``: sha256 of the oracle's surviving-vertex flags (uint8[n]).
* ``kept_sha256``: sha256 of the surviving edges, canonical and sorted (int32
  pairs), i.e. ``edges[elive]``.
* ``v_sweep_sha256``: sha256 of the 1-based productive sweep that deleted each
  vertex (int32[n], 0 = kept).
* ``sweeps``, ``passes``, ``tests``, ``dv``, ``de``, ``n_live``, ``m_live``.

Usage (from the repository root)::

    python tests/golden/make_full_size_digests.py c2 c3 c5c c4 --jobs 6

The Jacobi fixpoint of Section 4.2 is single-threaded in the oracle; ``--jobs``
only runs different graphs side by side (the batch's 1024 graphs, or the
single-graph workloads against each other).  Processes are spawned, not
forked.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "full_size")

BATCH_COUNT = 1024


def _sha(*arrays) -> str:
    import numpy as np
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()


def input_digest(colour, edges) -> str:
    import numpy as np
    return _sha(np.asarray(colour, dtype=np.int32), np.asarray(edges, dtype=np.int32).reshape(-1, 2))


def _record(g, short: bool = False) -> dict:
    import numpy as np
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import oracle
    edges = g.get_edges()
    t0 = time.time()
    orc = oracle.fixpoint(g.colour, edges, g.k)
    secs = time.time() - t0
    kept = np.ascontiguousarray(edges[orc["elive"].astype(bool)], dtype=np.int32)
    cut = (lambda s: s[:24]) if short else (lambda s: s)
    return dict(
        n=int(g.n), k=int(g.k), m=int(len(edges)),
        input_sha256=cut(input_digest(g.colour, edges)),
        vlive_sha256=cut(_sha(orc["vlive"].astype(np.uint8))),
        kept_sha256=cut(_sha(kept)),
        v_sweep_sha256=cut(_sha(orc["v_sweep"].astype(np.int32))),
        sweeps=int(orc["sweeps"]), passes=int(orc["passes"]), tests=int(orc["tests"]),
        dv=[int(x) for x in orc["dv"]], de=[int(x) for x in orc["de"]],
        n_live=int(orc["vlive"].sum()), m_live=int(len(kept)),
        oracle_seconds=round(secs, 1),
    )


def _single(name: str) -> tuple:
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2212_00574_gb300 import synth
    g = synth.workload(name)
    rec = _record(g)
    rec["workload"] = name
    rec["recipe"] = synth.WORKLOADS[name]
    rec["seed"] = synth.workload_seed(name)
    return name, rec


def _batch_item(j: int) -> tuple:
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2212_00574_gb300 import synth
    n, k, p, planted, seed = synth.batch_specs(BATCH_COUNT, synth.SEED_BASE + 4)[j]
    g = synth.kpartite(n, k, p, seed, planted=planted)
    rec = _record(g, short=True)
    rec.update(index=j, p=p, planted=planted, seed=seed)
    return j, rec


def _write(name: str, obj) -> None:
    os.makedirs(OUT, exist_ok=True)
    path = os.path.join(OUT, f"{name}.json")
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        if "graphs" in obj:  # the batch: one record per graph, kept compact
            json.dump(obj, f, sort_keys=True, separators=(",", ":"))
        else:
            json.dump(obj, f, indent=1, sort_keys=True)
        f.write("\n")
    os.replace(tmp, path)
    print(f"wrote {path}", flush=True)


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("workloads", nargs="+", choices=["c1", "c2", "c3", "c5c", "c4"])
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 2))
    a = ap.parse_args(argv)
    ctx = mp.get_context("spawn")
    singles = [w for w in a.workloads if w != "c4"]
    with ctx.Pool(a.jobs) as pool:
        # each single-graph record is written as soon as it is ready
        pending = [pool.apply_async(_single, (w,), callback=lambda r: _write(*r)) for w in singles]
        batch = {}
        if "c4" in a.workloads:
            # longest graphs first so the pool drains evenly
            from paper_2212_00574_gb300 import synth
            specs = synth.batch_specs(BATCH_COUNT, synth.SEED_BASE + 4)
            order = sorted(range(BATCH_COUNT), key=lambda j: -(specs[j][0] ** 3 * specs[j][2] ** 2))
            for j, rec in pool.imap_unordered(_batch_item, order):
                batch[j] = rec
                if len(batch) % 64 == 0:
                    print(f"c4: {len(batch)}/{BATCH_COUNT}", flush=True)
            _write("c4", dict(workload="c4", recipe=synth.WORKLOADS["c4"], seed=synth.SEED_BASE + 4,
                              count=BATCH_COUNT, digest_hex_chars=24,
                              graphs=[batch[j] for j in range(BATCH_COUNT)]))
        for p in pending:
            p.get()


if __name__ == "__main__":
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    main()
