"""Host logic of the benchmark and of the learned schedule's training set (CPU
only: no kernel runs here)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2212_00574_gb300 import learned, synth  # noqa: E402


def test_kernel_source_lists_exist():
    for kernel, files in bench.KERNEL_SOURCES.items():
        assert files, kernel
        for f in files:
            assert os.path.isfile(os.path.join(ROOT, "paper_2212_00574_gb300", "csrc", f)), (kernel, f)


def test_traffic_records_parse_and_match_the_sources():
    recs = bench.traffic_records()
    assert len(recs) >= 3
    for rec in recs:
        assert rec["kernel"] in bench.KERNEL_SOURCES, rec
        assert int(rec["dram_bytes_per_launch"]) > 0
        assert len(rec["sources_sha256"]) == 64
        assert rec["file"].startswith("profiles" + os.sep) or rec["file"].startswith("profiles/")
    # the benchmark's headline kernel has a record for its current sources
    got, src = bench.measured_traffic("c5", "bitset_persistent_kernel")
    assert got is not None and got > 135e6 and src.endswith(".md")


def test_traffic_lookup_needs_the_current_sources(tmp_path, monkeypatch):
    # a record whose hash does not match the kernel's sources is not used
    body = "```traffic-record\nworkload: w\nkernel: tensor_edge_kernel\nsources_sha256: " + "0" * 64 + \
           "\ndram_bytes_per_launch: 123\n```\n"
    (tmp_path / "x.md").write_text(body)
    monkeypatch.setattr(bench, "PROFILES", str(tmp_path))
    assert bench.measured_traffic("w", "tensor_edge_kernel") == (None, None)
    good = body.replace("0" * 64, bench.sources_sha256(bench.KERNEL_SOURCES["tensor_edge_kernel"]))
    (tmp_path / "x.md").write_text(good)
    assert bench.measured_traffic("w", "tensor_edge_kernel")[0] == 123.0
    assert bench.measured_traffic("w", "no_such_kernel") == (None, None)


def test_mlp_flops_per_edge():
    # two hidden layers of 64 and one output, multiply-adds counted twice
    assert bench.MLP_FLOPS_PER_EDGE == 2 * (16 * 64 + 64 * 64 + 64) == 10368


def test_cascade_specs_cover_the_regime():
    specs = learned.cascade_specs(200, 5)
    n = np.array([s[0] for s in specs])
    k = np.array([s[1] for s in specs])
    p = np.array([s[2] for s in specs])
    assert n.min() >= 256 and n.max() <= 32768 and n.max() > 8 * n.min()
    assert k.min() >= 8 and k.max() <= 32
    # an edge expects p^2 n / k common neighbours per class: 3 to 9 unless clipped
    mu = p * p * n / k
    unclipped = (p > 0.02) & (p < 0.6)
    assert np.all((mu[unclipped] > 3 - 1e-9) & (mu[unclipped] < 9 + 1e-9))
    assert [s[3] for s in specs[:4]] == [True, False, True, False]
    assert len({s[4] for s in specs}) == len(specs)
    assert learned.cascade_specs(10, 5) == learned.cascade_specs(10, 5)[:10]


def test_workload_seeds_are_distinct_and_recorded():
    names = ["c1", "c2", "c3", "c4", "c5", "c5c", "c5s"]
    seeds = [synth.workload_seed(w) for w in names]
    assert len(set(seeds)) == len(seeds)
    for w in names:
        assert w in bench.WORKLOAD_DESC
