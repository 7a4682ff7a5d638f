"""The C ABI on the CPU: the library loads, exports every function that
include/kz.h declares, and rejects bad input on the host before any CUDA
call.  No compute call is made here (no GPU in this environment)."""
import ctypes

import numpy as np
import pytest

import paper_2212_00574_gb300 as kz


@pytest.fixture(scope="module")
def lib():
    return kz._lib()


def test_header_symbols_exported(lib):
    names = kz.header_functions()
    assert {"kz_load_graph", "kz_kernelize", "kz_kernelize_batch", "kz_fetch_kernel"} <= set(names)
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/kz.h but not exported"


def test_struct_sizes_match_header():
    # kz_options: 2 x int32, int64, int32, 9 x int32 -> 56 bytes; kz_stats: 7 x int64 + 8 x int32
    assert ctypes.sizeof(kz.kz_options) == 56
    assert ctypes.sizeof(kz.kz_stats) == 7 * 8 + 8 * 4


def test_status_strings(lib):
    for code, name in kz.STATUS_NAMES.items():
        s = kz.kz_status_string(code)
        assert s and s != "unknown status", name
    assert kz.kz_status_string(999) == "unknown status"
    assert kz.kz_version() >= 100


def test_default_options():
    o = kz.kz_default_options()
    assert o.path == kz.PATHS["auto"] and o.schedule == 0 and o.use_graph == 1 and o.max_sweeps == 0


@pytest.mark.parametrize("colour,edges,k,code", [
    ([0, 0], [[0, 1]], 2, kz.KZ_ERR_ILLEGAL_COLOURING),
    ([0, 1], [[1, 1]], 2, kz.KZ_ERR_SELF_LOOP),
    ([0, 2], [[0, 1]], 2, kz.KZ_ERR_COLOUR_RANGE),
    ([0, -1], [[0, 1]], 2, kz.KZ_ERR_COLOUR_RANGE),
    ([0, 1], [[0, 7]], 2, kz.KZ_ERR_VERTEX_RANGE),
    ([0, 1], [[-1, 0]], 2, kz.KZ_ERR_VERTEX_RANGE),
    ([0, 1], [[0, 1]], 0, kz.KZ_ERR_ARG),
    ([0, 1], [[0, 1]], 65, kz.KZ_ERR_ARG),
])
def test_host_validation(colour, edges, k, code):
    with pytest.raises(kz.KzError) as ei:
        kz.kz_load_graph(len(colour), k, colour, edges)
    assert ei.value.status == code


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    col = np.zeros(3, np.int32)
    assert lib.kz_load_graph(3, 2, None, 0, None, 0, None, ctypes.byref(h)) == kz.KZ_ERR_ARG
    assert lib.kz_load_graph(3, 2, col.ctypes.data, 1, None, 0, None, ctypes.byref(h)) == kz.KZ_ERR_ARG
    assert lib.kz_load_graph(3, 2, col.ctypes.data, 0, None, 0, None, None) == kz.KZ_ERR_ARG
    assert lib.kz_load_graph(3, 2, col.ctypes.data, 0, None, 0x80, None, ctypes.byref(h)) == kz.KZ_ERR_ARG
    assert lib.kz_kernelize(None, None, None) == kz.KZ_ERR_ARG
    assert lib.kz_fetch_stats(None, None) == kz.KZ_ERR_ARG
    assert lib.kz_reset(None, None) == kz.KZ_ERR_ARG
    assert lib.kz_kernelize_batch(None, 2, None, None) == kz.KZ_ERR_ARG
    assert lib.kz_load_graph_dense(3, 2, col.ctypes.data, None, 1, 0, None, ctypes.byref(h)) == kz.KZ_ERR_ARG
    lib.kz_free_graph(None)  # ignored


def test_dense_row_words_checked(lib):
    h = ctypes.c_void_p()
    col = np.zeros(130, np.int32)
    bits = np.zeros((130, 2), np.uint64)
    # 130 vertices need 3 words per row
    assert lib.kz_load_graph_dense(130, 2, col.ctypes.data, bits.ctypes.data, 2, 0, None,
                                   ctypes.byref(h)) == kz.KZ_ERR_ARG


def test_no_cpu_fallback():
    """Valid input on a machine without a usable GPU fails loudly."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(kz.KzError) as ei:
        kz.kz_load_graph(2, 2, [0, 1], [[0, 1]])
    assert ei.value.status == kz.KZ_ERR_CUDA


def _header_struct_fields(name):
    import re
    src = open(kz.HEADER).read()
    end = re.search(r"\}\s*" + name + ";", src).start()
    body = src[src.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):  # "int64_t n, m" declares two fields
        if decl.strip():
            names += [re.sub(r"\[.*?\]", "", part).split()[-1] for part in decl.split(",")]
    return names


@pytest.mark.parametrize("name,cls", [("kz_options", kz.kz_options), ("kz_stats", kz.kz_stats)])
def test_struct_fields_follow_header(name, cls):
    # the binding's field order is the header's (offsets follow from it)
    assert [f for f, _ in cls._fields_] == _header_struct_fields(name)


def test_new_entry_points_validate_on_host(lib):
    found = ctypes.c_int32(0)
    q = ctypes.c_int32(0)
    out = (ctypes.c_int32 * 4)()
    assert lib.kz_find_clique(None, 3, 0, out, ctypes.byref(found)) == kz.KZ_ERR_ARG
    assert lib.kz_max_clique(None, None, 0, ctypes.byref(q), out, None) == kz.KZ_ERR_ARG
    d1, d2 = ctypes.c_double(), ctypes.c_double()
    assert lib.kz_probe_int_throughput(5, ctypes.byref(d1), ctypes.byref(d2), None) == kz.KZ_ERR_ARG
    assert lib.kz_probe_int_throughput(0, None, ctypes.byref(d2), None) == kz.KZ_ERR_ARG
    lib.kz_set_batch_tuning.argtypes = [ctypes.c_double, ctypes.c_int32, ctypes.c_int32]
    assert lib.kz_set_batch_tuning(float("nan"), 0, 0) == kz.KZ_ERR_ARG
    assert lib.kz_set_batch_tuning(0.0, 0, 0) == kz.KZ_OK   # the defaults
