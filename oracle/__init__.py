"""CPU oracle for the colour-index kernelization (thesis Section 4.2).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the CPU
baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or runs anything under ``oracle/``.

The arithmetic lives in ``kz_oracle.c`` (plain single-threaded C, compiled
with gcc on first use into ``oracle/_build/``).  This module only marshals
arguments.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kz_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libkzoracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {
    0: "ok",
    -1: "bad argument",
    -2: "colour out of range",
    -3: "illegal colouring",
    -4: "self loop",
    -5: "vertex out of range",
    -6: "out of memory",
    -7: "sweep limit reached",
}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, '?')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: no -march)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source (used by the tests that
    check that the pins catch plausible mistakes)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-w", "-shared", "-fPIC", "-o", out_path, src])
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _bind(path: str):
    lib = C.CDLL(path)
    P = C.c_void_p
    i32, i64 = C.c_int32, C.c_int64
    lib.kzo_fixpoint.restype = C.c_int
    lib.kzo_fixpoint.argtypes = [i32, i32, P, i64, P, i64, P, P, P, P, P, P, i64, P, P]
    lib.kzo_fixpoint_dominance.restype = C.c_int
    lib.kzo_fixpoint_dominance.argtypes = [i32, i32, i32, P, i64, P, P, P, P, P]
    lib.kzo_fixpoint_edge_dominance.restype = C.c_int
    lib.kzo_fixpoint_edge_dominance.argtypes = [i32, i32, i32, P, i64, P, P, P, P, P]
    lib.kzo_fixpoint_q.restype = C.c_int
    lib.kzo_fixpoint_q.argtypes = [i32, i32, i32, P, i64, P, i64, P, P, P, P, P, P, i64, P, P]
    lib.kzo_indices.restype = C.c_int
    lib.kzo_indices.argtypes = [i32, i32, P, i64, P, P, P, P, i64, P, P, i64, P]
    lib.kzo_dense_indices.restype = C.c_int
    lib.kzo_dense_indices.argtypes = [i32, i32, P, P, i64, P, P, i64, P, P, i64, P]
    lib.kzo_open.restype = C.c_void_p
    lib.kzo_open.argtypes = [i32, i32, P, i64, P, P]
    lib.kzo_session_edge_index.restype = C.c_int
    lib.kzo_session_edge_index.argtypes = [P, P, i64, P]
    lib.kzo_close.restype = None
    lib.kzo_close.argtypes = [P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


class Oracle:
    """The oracle's functions bound to one compiled library (the default
    build, or an edited variant for mutation tests)."""

    def __init__(self, lib_path: str | None = None):
        self._lib = _bind(lib_path) if lib_path else None

    def lib(self):
        return self._lib if self._lib is not None else _load()

    def fixpoint(self, *a, **kw):
        return fixpoint(*a, _lib=self.lib(), **kw)

    def fixpoint_dominance(self, *a, **kw):
        return fixpoint_dominance(*a, _lib=self.lib(), **kw)

    def fixpoint_edge_dominance(self, *a, **kw):
        return fixpoint_edge_dominance(*a, _lib=self.lib(), **kw)

    def indices(self, *a, **kw):
        return indices(*a, _lib=self.lib(), **kw)

    def dense_indices(self, *a, **kw):
        return dense_indices(*a, _lib=self.lib(), **kw)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def fixpoint_dominance(colour, edges, k: int, clique_k: int | None = None, _lib=None) -> dict:
    """Colour-index fixpoint, then rounds of vertex dominance (Definition
    4.3.1), each followed by the colour-index fixpoint again, until a round
    deletes nothing.  Returns ``vlive``, ``elive``, ``rounds`` (dominance
    rounds that deleted something) and ``dominated`` (vertices they deleted)."""
    lib = _lib or _load()
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    edges = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    n, m = len(colour), len(edges)
    vlive = np.zeros(n, np.uint8)
    elive = np.zeros(m, np.uint8)
    rounds, dominated = C.c_int64(0), C.c_int64(0)
    q = int(k if clique_k is None else clique_k)
    rc = lib.kzo_fixpoint_dominance(n, int(k), q, _ptr(colour), m, _ptr(edges), _ptr(vlive), _ptr(elive),
                                    C.addressof(rounds), C.addressof(dominated))
    if rc != 0:
        raise OracleError(rc)
    return dict(vlive=vlive, elive=elive, rounds=int(rounds.value), dominated=int(dominated.value))


def fixpoint_edge_dominance(colour, edges, k: int, clique_k: int | None = None, _lib=None) -> dict:
    """Colour-index fixpoint, then rounds of edge dominance (Definitions 4.3.2
    and 4.3.3), each followed by the colour-index fixpoint again, until a
    round deletes nothing.  Returns ``vlive``, ``elive``, ``rounds`` (rounds
    that deleted something) and ``deleted`` (edges they deleted).  n <= 4096."""
    lib = _lib or _load()
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    edges = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    n, m = len(colour), len(edges)
    vlive = np.zeros(n, np.uint8)
    elive = np.zeros(m, np.uint8)
    rounds, deleted = C.c_int64(0), C.c_int64(0)
    q = int(k if clique_k is None else clique_k)
    rc = lib.kzo_fixpoint_edge_dominance(n, int(k), q, _ptr(colour), m, _ptr(edges), _ptr(vlive), _ptr(elive),
                                         C.addressof(rounds), C.addressof(deleted))
    if rc != 0:
        raise OracleError(rc)
    return dict(vlive=vlive, elive=elive, rounds=int(rounds.value), deleted=int(deleted.value))


def fixpoint(colour, edges, k: int, max_sweeps: int = 0, raise_on_limit: bool = True, _lib=None,
             clique_k: int | None = None) -> dict:
    """Jacobi fixpoint of the vertex and edge colour-index rules.

    ``clique_k`` is the clique size q sought (default k): a vertex fails below
    colour index q-1 and an edge below q-2 (Section 4.2, Remarks).

    Returns a dict with ``vlive`` (uint8[n]), ``elive`` (uint8[m], input edge
    order), ``v_sweep`` / ``e_rule_sweep`` (int32, 1-based productive sweep
    of deletion, 0 = never), ``dv`` / ``de`` (per productive sweep counts),
    ``sweeps``, ``passes`` (= sweeps + 1 unless the limit stopped it),
    ``tests`` (live edges tested over all passes) and ``status``.
    """
    lib = _lib or _load()
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    edges = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    n, m = len(colour), len(edges)
    cap = n + m + 2
    vlive = np.zeros(n, np.uint8)
    elive = np.zeros(m, np.uint8)
    v_sweep = np.zeros(n, np.int32)
    e_rule = np.zeros(m, np.int32)
    dv = np.zeros(cap, np.int64)
    de = np.zeros(cap, np.int64)
    sweeps = C.c_int64(0)
    tests = C.c_int64(0)
    q = int(k if clique_k is None else clique_k)
    rc = lib.kzo_fixpoint_q(n, int(k), q, _ptr(colour), m, _ptr(edges), int(max_sweeps),
                          _ptr(vlive), _ptr(elive), _ptr(v_sweep), _ptr(e_rule),
                          _ptr(dv), _ptr(de), cap, C.addressof(sweeps), C.addressof(tests))
    if rc not in (0, -7) or (rc == -7 and raise_on_limit):
        raise OracleError(rc)
    s = int(sweeps.value)
    return dict(vlive=vlive, elive=elive, v_sweep=v_sweep, e_rule_sweep=e_rule,
                dv=dv[:s].copy(), de=de[:s].copy(), sweeps=s,
                passes=s + 1 if rc == 0 else s, tests=int(tests.value), status=rc)


def indices(colour, edges, k: int, verts=(), edge_ids=(), vlive=None, elive=None, _lib=None):
    """Vertex and edge colour indices (Section 4.2) on a live state."""
    lib = _lib or _load()
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    edges = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
    verts = np.ascontiguousarray(verts, dtype=np.int32)
    edge_ids = np.ascontiguousarray(edge_ids, dtype=np.int64)
    vl = None if vlive is None else np.ascontiguousarray(vlive, dtype=np.uint8)
    el = None if elive is None else np.ascontiguousarray(elive, dtype=np.uint8)
    out_v = np.zeros(len(verts), np.int32)
    out_e = np.zeros(len(edge_ids), np.int32)
    rc = lib.kzo_indices(len(colour), int(k), _ptr(colour), len(edges), _ptr(edges), _ptr(vl), _ptr(el),
                         _ptr(verts), len(verts), _ptr(out_v), _ptr(edge_ids), len(edge_ids), _ptr(out_e))
    if rc != 0:
        raise OracleError(rc)
    return out_v, out_e


def dense_indices(colour, bits, k: int, verts=(), pairs=(), vlive=None, _lib=None):
    """Colour indices read off a dense uint64 bit adjacency matrix."""
    lib = _lib or _load()
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    bits = np.ascontiguousarray(bits, dtype=np.uint64)
    n = len(colour)
    verts = np.ascontiguousarray(verts, dtype=np.int32)
    pairs = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
    vl = None if vlive is None else np.ascontiguousarray(vlive, dtype=np.uint8)
    out_v = np.zeros(len(verts), np.int32)
    out_e = np.zeros(len(pairs), np.int32)
    rc = lib.kzo_dense_indices(n, int(k), _ptr(colour), _ptr(bits), bits.shape[1], _ptr(vl),
                               _ptr(verts), len(verts), _ptr(out_v), _ptr(pairs), len(pairs), _ptr(out_e))
    if rc != 0:
        raise OracleError(rc)
    return out_v, out_e


class Session:
    """Edge colour indices of one graph, queried repeatedly (adjacency built
    once).  Every element is live."""

    def __init__(self, colour, edges, k: int, _lib=None):
        self._lib = _lib or _load()
        self.colour = np.ascontiguousarray(colour, dtype=np.int32)
        self.edges = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        rc = C.c_int(0)
        self.h = self._lib.kzo_open(len(self.colour), int(k), _ptr(self.colour), len(self.edges),
                                    _ptr(self.edges), C.byref(rc))
        if not self.h:
            raise OracleError(rc.value)

    def edge_index(self, edge_ids) -> np.ndarray:
        ids = np.ascontiguousarray(edge_ids, dtype=np.int64)
        out = np.zeros(len(ids), np.int32)
        rc = self._lib.kzo_session_edge_index(self.h, _ptr(ids), len(ids), _ptr(out))
        if rc != 0:
            raise OracleError(rc)
        return out

    def close(self):
        if self.h:
            self._lib.kzo_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
