"""Python binding of libkz.so, the GB300 colour-index kernelization library.

The functions here carry the C ABI's names (``kz_load_graph``,
``kz_kernelize``, ``kz_kernelize_batch``, ``kz_fetch_kernel`` ...) and only
marshal arguments: every step of the method runs in the library's CUDA
kernels.  There is no CPU fallback; without the built library or a GPU the
calls raise.

Device memory for graph handles comes from PyTorch's caching allocator when
PyTorch with CUDA is available (``use_torch_allocator``); streams are raw
``cudaStream_t`` values (``torch.cuda.current_stream().cuda_stream`` by
default).
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

from . import build as _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "kz.h")
HEADERS = [HEADER, os.path.join(os.path.dirname(HEADER), "kz_probe.h"),
           os.path.join(os.path.dirname(HEADER), "kz_learned.h")]

KZ_OK = 0
STATUS_NAMES = {
    0: "KZ_OK", 1: "KZ_ERR_ARG", 2: "KZ_ERR_COLOUR_RANGE", 3: "KZ_ERR_ILLEGAL_COLOURING",
    4: "KZ_ERR_SELF_LOOP", 5: "KZ_ERR_VERTEX_RANGE", 6: "KZ_ERR_DUPLICATE_EDGE", 7: "KZ_ERR_OOM",
    8: "KZ_ERR_CUDA", 9: "KZ_ERR_LIMIT", 10: "KZ_ERR_TIMEOUT", 11: "KZ_ERR_NOT_READY",
    12: "KZ_ERR_BUFFER", 13: "KZ_ERR_UNSUPPORTED", 14: "KZ_ERR_INTERNAL",
}
globals().update({v: k for k, v in STATUS_NAMES.items()})

KZ_DEDUP = 0x1
PATHS = {"auto": 0, "bitset": 1, "small": 2, "sparse": 3, "tensor": 4}
SCHEDULES = {"plain": 0, "learned": 1, "support": 2}
PLANE0 = {"auto": 0, "full": 1, "half": 2, "two": 3}
BATCH = {"concurrent": 0, "sequential": 1, "fused": 2}


class KzError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        name = STATUS_NAMES.get(self.status, str(status))
        msg = _lib().kz_status_string(self.status).decode() if _LIB is not None else ""
        super().__init__(f"{where}: {name} ({msg})")


class kz_options(C.Structure):
    _fields_ = [("path", C.c_int32), ("schedule", C.c_int32), ("max_sweeps", C.c_int64),
                ("use_graph", C.c_int32), ("plane0", C.c_int32), ("batch", C.c_int32),
                ("clique_k", C.c_int32), ("dominance", C.c_int32), ("tensor_precision", C.c_int32),
                ("reserved", C.c_int32 * 4)]


class kz_stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("n_live", C.c_int64), ("m_live", C.c_int64),
                ("sweeps", C.c_int64), ("passes", C.c_int64), ("edge_tests", C.c_int64),
                ("path", C.c_int32), ("status", C.c_int32), ("k", C.c_int32), ("clique_k", C.c_int32),
                ("dominance_rounds", C.c_int32), ("dominated", C.c_int32), ("reserved", C.c_int32 * 2)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class kz_allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


_LIB = None
_LOCK = threading.Lock()


def library_path() -> str:
    return _build.LIB


def _lib():
    """Load libkz.so (building it first when the sources are newer)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.build() if _build.stale() else _build.LIB
            lib = C.CDLL(path)
            P, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
            sig = {
                "kz_default_options": (None, [P]),
                "kz_set_allocator": (C.c_int, [P]),
                "kz_load_graph": (C.c_int, [i32, i32, P, i64, P, u32, P, P]),
                "kz_load_graph_dense": (C.c_int, [i32, i32, P, P, i64, u32, P, P]),
                "kz_kernelize": (C.c_int, [P, P, P]),
                "kz_kernelize_batch": (C.c_int, [P, i32, P, P]),
                "kz_fetch_kernel": (C.c_int, [P, P, P, i64, P, P]),
                "kz_fetch_kernel_dense": (C.c_int, [P, P, P, i64, P]),
                "kz_fetch_stats": (C.c_int, [P, P]),
                "kz_fetch_trace": (C.c_int, [P, P, P, i64, P]),
                "kz_reset": (C.c_int, [P, P]),
                "kz_free_graph": (None, [P]),
                "kz_status_string": (C.c_char_p, [C.c_int]),
                "kz_version": (i32, []),
                "kz_probe_int_throughput": (C.c_int, [i32, P, P, P]),
                "kz_set_batch_tuning": (C.c_int, [C.c_double, i32, i32]),
                "kz_find_clique": (C.c_int, [P, i32, i64, P, P]),
                "kz_max_clique": (C.c_int, [P, P, i64, P, P, P]),
                "kz_probe_barrier_timeout": (C.c_int, [P, u32, P]),
                "kz_kernelize_dense_noalloc": (C.c_int, [i32, i32, P, P, i64, i64, P, P, P, P]),
                "kz_model_create": (C.c_int, [P, P]),
                "kz_model_get": (C.c_int, [P, P]),
                "kz_model_free": (None, [P]),
                "kz_mlp_forward": (C.c_int, [P, P, i64, P, P]),
                "kz_mlp_grad": (C.c_int, [P, P, P, i64, P, P, P]),
                "kz_mlp_adam": (C.c_int, [P, P, C.c_float, P]),
                "kz_collect_trace": (C.c_int, [P, i64, C.c_uint64, P, P, i64, P]),
                "kz_attach_model": (C.c_int, [P, P, C.c_float]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _LIB = lib
    return _LIB


def header_functions() -> list:
    """Names of the functions declared in the headers under include/."""
    names = set()
    for h in HEADERS:
        with open(h) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(kz_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(status: int, where: str):
    if status != KZ_OK:
        raise KzError(status, where)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# ---------------------------------------------------------------------------
# allocator: PyTorch's caching allocator behind the C callbacks
# ---------------------------------------------------------------------------

_TORCH_ALLOC = None


def use_torch_allocator() -> bool:
    """Route the library's device allocations through torch's caching
    allocator.  Returns False (and leaves cudaMallocAsync in place) when torch
    has no CUDA device."""
    global _TORCH_ALLOC
    try:
        import torch
    except Exception:
        return False
    if not torch.cuda.is_available():
        return False
    if _TORCH_ALLOC is not None:
        return True

    def _alloc(nbytes, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          int(stream or 0)))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    a = kz_allocator(_ALLOC_FN(_alloc), _FREE_FN(_free), None)
    _check(_lib().kz_set_allocator(C.byref(a)), "kz_set_allocator")
    _TORCH_ALLOC = a  # keep the callbacks alive
    return True


def use_default_allocator():
    global _TORCH_ALLOC
    _check(_lib().kz_set_allocator(None), "kz_set_allocator")
    _TORCH_ALLOC = None


# ---------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------

def kz_default_options(**kw) -> kz_options:
    o = kz_options()
    _lib().kz_default_options(C.byref(o))
    for key, val in kw.items():
        if key == "path" and isinstance(val, str):
            val = PATHS[val]
        if key == "schedule" and isinstance(val, str):
            val = SCHEDULES[val]
        if key == "plane0" and isinstance(val, str):
            val = PLANE0[val]
        if key == "batch" and isinstance(val, str):
            val = BATCH[val]
        setattr(o, key, int(val))
    return o


def kz_load_graph(n: int, k: int, colour, edges, flags: int = 0, stream=None) -> int:
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    edges = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    if len(colour) != n:
        raise ValueError("colour must have n entries")
    h = C.c_void_p()
    st = _lib().kz_load_graph(int(n), int(k), _ptr(colour), len(edges), _ptr(edges), int(flags),
                              _stream(stream), C.byref(h))
    _check(st, "kz_load_graph")
    return h.value


def kz_load_graph_dense(n: int, k: int, colour, adj_bits, flags: int = 0, stream=None) -> int:
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    bits = np.ascontiguousarray(adj_bits, dtype=np.uint64)
    if bits.ndim != 2 or bits.shape[0] != n:
        raise ValueError("adj_bits must be uint64[n, row_words]")
    h = C.c_void_p()
    st = _lib().kz_load_graph_dense(int(n), int(k), _ptr(colour), _ptr(bits), bits.shape[1], int(flags),
                                    _stream(stream), C.byref(h))
    _check(st, "kz_load_graph_dense")
    return h.value


def kz_kernelize(g: int, options: kz_options | None = None, stream=None):
    st = _lib().kz_kernelize(C.c_void_p(g), None if options is None else C.byref(options), _stream(stream))
    _check(st, "kz_kernelize")


def kz_kernelize_batch(graphs, options: kz_options | None = None, stream=None):
    arr = (C.c_void_p * len(graphs))(*[C.c_void_p(h) for h in graphs])
    st = _lib().kz_kernelize_batch(arr, len(graphs), None if options is None else C.byref(options),
                                   _stream(stream))
    _check(st, "kz_kernelize_batch")


def kz_set_batch_tuning(group_spread: float = 0.0, items_per_warp: int = 0, max_group: int = 0):
    """Tuning of the fused batch's cost model (0 restores a default)."""
    _check(_lib().kz_set_batch_tuning(float(group_spread), int(items_per_warp), int(max_group)),
           "kz_set_batch_tuning")


def kz_fetch_stats(g: int, allow=(KZ_OK,)) -> dict:
    s = kz_stats()
    st = _lib().kz_fetch_stats(C.c_void_p(g), C.byref(s))
    if st not in allow:
        raise KzError(st, "kz_fetch_stats")
    return s.as_dict()


def kz_fetch_kernel(g: int, n: int, cap: int | None = None, allow=(KZ_OK,)):
    """Returns (vertex_alive uint8[n], edges int32[m_live, 2], stats dict)."""
    alive = np.zeros(n, np.uint8)
    m_out = C.c_int64(0)
    s = kz_stats()
    if cap is None:
        st = _lib().kz_fetch_stats(C.c_void_p(g), C.byref(s))
        if st not in allow:
            raise KzError(st, "kz_fetch_kernel")
        cap = max(int(s.m), 0)
    edges = np.zeros((max(cap, 1), 2), np.int32)
    st = _lib().kz_fetch_kernel(C.c_void_p(g), _ptr(alive), _ptr(edges), int(cap), C.byref(m_out), C.byref(s))
    if st not in allow:
        raise KzError(st, "kz_fetch_kernel")
    d = s.as_dict()
    d["m_live"] = int(m_out.value)
    return alive, edges[:int(m_out.value)].copy(), d


def kz_fetch_kernel_dense(g: int, n: int, allow=(KZ_OK,), out_bits=None, out_alive=None):
    """Returns (vertex_alive uint8[n], bits uint64[n, row_words], stats dict).
    ``out_bits`` / ``out_alive`` may be given (for example pinned buffers)."""
    alive = np.zeros(n, np.uint8) if out_alive is None else out_alive
    bits = np.zeros((n, max((n + 63) // 64, 1)), np.uint64) if out_bits is None else out_bits
    if bits.dtype != np.uint64 or not bits.flags.c_contiguous or bits.shape[0] != n:
        raise ValueError("out_bits must be a C-contiguous uint64[n, row_words] array")
    if alive.dtype != np.uint8 or len(alive) != n:
        raise ValueError("out_alive must be uint8[n]")
    s = kz_stats()
    st = _lib().kz_fetch_kernel_dense(C.c_void_p(g), _ptr(alive), _ptr(bits), bits.shape[1], C.byref(s))
    if st not in allow:
        raise KzError(st, "kz_fetch_kernel_dense")
    return alive, bits, s.as_dict()


def kz_fetch_trace(g: int, n: int, cap: int = 1 << 16):
    dv = np.zeros(cap, np.int64)
    de = np.zeros(cap, np.int64)
    vs = np.zeros(n, np.int32)
    _check(_lib().kz_fetch_trace(C.c_void_p(g), _ptr(dv), _ptr(de), cap, _ptr(vs)), "kz_fetch_trace")
    return dv, de, vs


def kz_reset(g: int, stream=None):
    _check(_lib().kz_reset(C.c_void_p(g), _stream(stream)), "kz_reset")


def kz_free_graph(g: int):
    _lib().kz_free_graph(C.c_void_p(g))


def kz_status_string(status: int) -> str:
    return _lib().kz_status_string(int(status)).decode()


def kz_version() -> int:
    return int(_lib().kz_version())


def kz_kernelize_dense_noalloc(n: int, k: int, colour_ptr: int, adj_bits_ptr: int, row_words: int,
                               max_sweeps: int, alive_ptr: int, adj_out_ptr: int, counts_ptr: int,
                               stream=None) -> int:
    """Allocation-free kernelization of one graph; every pointer is a device
    address owned by the caller.  Returns the status (not raised: KZ_ERR_LIMIT
    still leaves a valid partial kernel)."""
    return int(_lib().kz_kernelize_dense_noalloc(int(n), int(k), C.c_void_p(colour_ptr),
                                                 C.c_void_p(adj_bits_ptr), int(row_words),
                                                 int(max_sweeps), C.c_void_p(alive_ptr),
                                                 C.c_void_p(adj_out_ptr), C.c_void_p(counts_ptr),
                                                 _stream(stream)))


def kz_probe_barrier_timeout(g: int, spin_limit: int = 1 << 14, stream=None):
    _check(_lib().kz_probe_barrier_timeout(C.c_void_p(g), int(spin_limit), _stream(stream)),
           "kz_probe_barrier_timeout")


def kz_find_clique(g: int, q: int, node_limit: int = 0):
    """(found, clique) on the current kernel: clique is int32[q] caller ids,
    ascending (empty when none was found)."""
    out = np.zeros(max(int(q), 1), np.int32)
    found = C.c_int32(0)
    _check(_lib().kz_find_clique(C.c_void_p(g), int(q), int(node_limit), _ptr(out), C.byref(found)),
           "kz_find_clique")
    return bool(found.value), (out[:q].copy() if found.value else np.zeros(0, np.int32))


def kz_max_clique(g: int, k: int, options: kz_options | None = None, node_limit: int = 0, stream=None):
    """(clique number, one maximum clique as ascending caller ids)."""
    out = np.zeros(max(int(k), 1), np.int32)
    q = C.c_int32(0)
    _check(_lib().kz_max_clique(C.c_void_p(g), None if options is None else C.byref(options), int(node_limit),
                                C.byref(q), _ptr(out), _stream(stream)), "kz_max_clique")
    return int(q.value), out[:q.value].copy()


def kz_probe_int_throughput(kind: int, stream=None):
    """(ops per second, kernel ms) of the integer-throughput probe."""
    ops = C.c_double(0)
    ms = C.c_double(0)
    _check(_lib().kz_probe_int_throughput(int(kind), C.byref(ops), C.byref(ms), _stream(stream)),
           "kz_probe_int_throughput")
    return ops.value, ms.value


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class KernelGraph:
    """Owns one kz_graph handle."""

    def __init__(self, n: int, k: int, colour, edges=None, bits=None, flags: int = 0, stream=None):
        self.n, self.k = int(n), int(k)
        if bits is not None:
            self.h = kz_load_graph_dense(n, k, colour, bits, flags, stream)
        else:
            self.h = kz_load_graph(n, k, colour, edges, flags, stream)

    @classmethod
    def from_synth(cls, g, dense: bool | None = None, stream=None):
        if dense is None:
            dense = g.bits is not None
        if dense:
            return cls(g.n, g.k, g.colour, bits=g.get_bits(), stream=stream)
        return cls(g.n, g.k, g.colour, edges=g.get_edges(), stream=stream)

    def kernelize(self, stream=None, **opts):
        kz_kernelize(self.h, kz_default_options(**opts), stream)
        return self

    def fetch(self, allow=(KZ_OK,)):
        return kz_fetch_kernel(self.h, self.n, allow=allow)

    def fetch_dense(self, allow=(KZ_OK,)):
        return kz_fetch_kernel_dense(self.h, self.n, allow=allow)

    def stats(self, allow=(KZ_OK,)):
        return kz_fetch_stats(self.h, allow=allow)

    def trace(self):
        return kz_fetch_trace(self.h, self.n)

    def reset(self, stream=None):
        kz_reset(self.h, stream)
        return self

    def close(self):
        if getattr(self, "h", None):
            kz_free_graph(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------
# learned schedule (include/kz_learned.h)
# ---------------------------------------------------------------------------

KZ_MLP_PARAMS = 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1


def kz_model_create(weights=None) -> int:
    h = C.c_void_p()
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    if w is not None and w.size != KZ_MLP_PARAMS:
        raise ValueError("weights must have KZ_MLP_PARAMS entries")
    _check(_lib().kz_model_create(_ptr(w), C.byref(h)), "kz_model_create")
    return h.value


def kz_model_get(m: int) -> np.ndarray:
    w = np.zeros(KZ_MLP_PARAMS, np.float32)
    _check(_lib().kz_model_get(C.c_void_p(m), _ptr(w)), "kz_model_get")
    return w


def kz_model_free(m: int):
    _lib().kz_model_free(C.c_void_p(m))


def kz_mlp_forward(m: int, X_ptr: int, B: int, logits_ptr: int, stream=None):
    _check(_lib().kz_mlp_forward(C.c_void_p(m), C.c_void_p(X_ptr), int(B), C.c_void_p(logits_ptr),
                                 _stream(stream)), "kz_mlp_forward")


def kz_mlp_grad(m: int, X_ptr: int, y_ptr: int, B: int, grad_ptr: int, loss_ptr: int, stream=None):
    _check(_lib().kz_mlp_grad(C.c_void_p(m), C.c_void_p(X_ptr), C.c_void_p(y_ptr), int(B), C.c_void_p(grad_ptr),
                              C.c_void_p(loss_ptr), _stream(stream)), "kz_mlp_grad")


def kz_mlp_adam(m: int, grad_ptr: int, lr: float, stream=None):
    _check(_lib().kz_mlp_adam(C.c_void_p(m), C.c_void_p(grad_ptr), C.c_float(lr), _stream(stream)), "kz_mlp_adam")


def kz_collect_trace(g: int, per_sweep_cap: int, seed: int, cap: int):
    """(features float32[count,16], labels uint8[count]) from plain sweeps."""
    X = np.zeros((max(cap, 1), 16), np.float32)
    y = np.zeros(max(cap, 1), np.uint8)
    cnt = C.c_int64(0)
    _check(_lib().kz_collect_trace(C.c_void_p(g), int(per_sweep_cap), C.c_uint64(seed), _ptr(X), _ptr(y), int(cap),
                                   C.byref(cnt)), "kz_collect_trace")
    return X[:cnt.value].copy(), y[:cnt.value].copy()


def kz_attach_model(g: int, m: int, threshold: float = 0.5):
    _check(_lib().kz_attach_model(C.c_void_p(g), C.c_void_p(m), C.c_float(threshold)), "kz_attach_model")
