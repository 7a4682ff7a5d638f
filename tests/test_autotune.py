"""The AUTO table compiled into kz_api.cu is the one the autotuner derives
from its recorded measurements (CPU only: no timing here)."""
import json
import os
import re

from paper_2212_00574_gb300 import autotune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _compiled_table():
    src = open(os.path.join(ROOT, "paper_2212_00574_gb300", "csrc", "kz_api.cu")).read()
    body = re.search(r"kTensorTable\[\d+\]\[2\]\[\d+\] = \{(.*?)\n\};", src, re.S).group(1)
    body = re.sub(r"//[^\n]*", "", body)
    nums = [int(x) for x in re.findall(r"\d+", body)]
    nd = len(autotune.D_EDGES) + 1
    return [[nums[(i * 2 + j) * nd:(i * 2 + j + 1) * nd] for j in range(2)] for i in range(len(nums) // (2 * nd))]


def test_compiled_table_matches_measurements():
    records = json.load(open(autotune.GRID_FILE))["records"]
    assert len(records) == 140
    assert autotune.table_from(records) == _compiled_table()


def test_cells_and_rendering():
    assert autotune.cell(2048, 12, 0.05) == (0, 0, 0)
    assert autotune.cell(32768, 24, 0.12) == (3, 1, 1)
    assert autotune.cell(4500, 12, 0.6) == (1, 0, 4)
    t = autotune.table_from([dict(n=8192, k=24, p=0.2, bitset_us=10, tensor_us=5)])
    assert t[2][1][2] == 1 and sum(map(sum, (r for per in t for r in per))) == 1
    assert "kTensorTable[4][2][5]" in autotune.render_c(t)


def test_bin_edges_match_the_library():
    src = open(os.path.join(ROOT, "paper_2212_00574_gb300", "csrc", "kz_api.cu")).read()
    body = src[src.index("static bool tensor_preferred"):src.index("static int auto_path")]
    nb = [int(x) for x in re.findall(r"g->n < (\d+)", body)]
    kb = [int(x) for x in re.findall(r"g->k < (\d+) \?", body)]
    db = [float(x) for x in re.findall(r"d < ([0-9.]+)", body)]
    assert tuple(nb) == autotune.N_EDGES and kb == [autotune.K_EDGE] and tuple(db) == autotune.D_EDGES


def test_batch_constants_match_measurements():
    records = json.load(open(autotune.BATCH_FILE))["records"]
    src = open(os.path.join(ROOT, "paper_2212_00574_gb300", "csrc", "kz_batch.cu")).read()
    assert autotune.render_batch_c(autotune.best_batch_tuning(records)) in src
