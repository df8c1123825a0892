"""Oracle for exact multiple-pattern matching — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package. The product path (the CUDA scan behind
``include/ac.h`` and its Python binding) never imports it.

A thin ctypes wrapper around ``ac_oracle.c`` (plain C, compiled with gcc):

* :func:`scan` — Aho-Corasick with failure links (Section II.A, Fig. 1);
* :func:`scan_mt` — the same machine over text chunks on POSIX threads,
  each chunk warmed up on the (longest pattern − 1) characters before it;
* :func:`pfac` — the failure-less walk from every start position
  (Section II.B, Figs. 2-4; Section IV.A, Fig. 6);
* :func:`brute` — the definition of the result set written out.

All return ``(matches, counts)``: ``matches`` is an ``(M, 2)`` uint32 array of
``(end position, pattern id)`` rows sorted by position then id (0-based,
inclusive end), ``counts`` a uint64 array with one entry per pattern.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "ac_oracle.c")
LIB = os.path.join(_HERE, "liboracle.so")

_lock = threading.Lock()
_lib = None


def build_oracle(out_path: str = LIB, mutant: int = 0) -> str:
    """Compile the oracle with gcc into ``out_path``.

    ``mutant`` > 0 compiles a deliberately broken variant (used by the tests
    that check that the pins catch plausible mistakes).
    """
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
           f"-DORACLE_MUTANT={int(mutant)}", SRC, "-o", out_path]
    subprocess.run(cmd, check=True, capture_output=True)
    return out_path


def _declare(lib):
    u32p = C.POINTER(C.c_uint32)
    lib.oracle_build.argtypes = [C.POINTER(C.c_void_p), u32p, C.c_uint32, C.c_int, C.POINTER(C.c_void_p)]
    lib.oracle_build.restype = C.c_int
    lib.oracle_free.argtypes = [C.c_void_p]
    lib.oracle_free.restype = None
    for name in ("oracle_num_states", "oracle_max_len"):
        getattr(lib, name).argtypes = [C.c_void_p]
        getattr(lib, name).restype = C.c_uint32
    for name in ("oracle_fail", "oracle_depth"):
        getattr(lib, name).argtypes = [C.c_void_p, C.c_uint32]
        getattr(lib, name).restype = C.c_uint32
    lib.oracle_goto.argtypes = [C.c_void_p, C.c_uint32, C.c_uint8]
    lib.oracle_goto.restype = C.c_uint32
    lib.oracle_state_of.argtypes = [C.c_void_p, C.c_char_p, C.c_uint32]
    lib.oracle_state_of.restype = C.c_uint32
    lib.oracle_trace.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, u32p]
    lib.oracle_trace.restype = C.c_int
    pp = C.POINTER(u32p)
    lib.oracle_scan.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, pp, C.POINTER(C.c_uint64)]
    lib.oracle_scan.restype = C.c_int
    lib.oracle_scan_mt.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int, pp, C.POINTER(C.c_uint64)]
    lib.oracle_scan_mt.restype = C.c_int
    lib.oracle_pfac.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, pp, C.POINTER(C.c_uint64)]
    lib.oracle_pfac.restype = C.c_int
    lib.oracle_pfac_walk.argtypes = [C.c_void_p, C.c_void_p, C.c_uint64, C.c_uint64, u32p, C.c_uint64]
    lib.oracle_pfac_walk.restype = C.c_uint64
    lib.oracle_brute.argtypes = [C.POINTER(C.c_void_p), u32p, C.c_uint32, C.c_void_p, C.c_uint64, pp,
                                 C.POINTER(C.c_uint64)]
    lib.oracle_brute.restype = C.c_int
    lib.oracle_counts.argtypes = [u32p, C.c_uint64, C.c_uint32, C.POINTER(C.c_uint64)]
    lib.oracle_counts.restype = None
    lib.oracle_free_buf.argtypes = [C.c_void_p]
    lib.oracle_free_buf.restype = None
    return lib


def load(path: str | None = None):
    """Load the oracle library (compiling it first if needed); ``path`` loads
    another build (e.g. a mutant) without caching it."""
    global _lib
    if path is not None:
        return _declare(C.CDLL(path))
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
                build_oracle()
            _lib = _declare(C.CDLL(LIB))
    return _lib


def _as_bytes(x) -> bytes:
    if isinstance(x, (bytes, bytearray)):
        return bytes(x)
    if isinstance(x, str):
        return x.encode()
    return np.asarray(x, dtype=np.uint8).tobytes()


def _text_buf(text):
    arr = np.ascontiguousarray(np.frombuffer(_as_bytes(text), dtype=np.uint8)) if not isinstance(
        text, np.ndarray) else np.ascontiguousarray(text, dtype=np.uint8)
    return arr, arr.ctypes.data_as(C.c_void_p), arr.size


def _pattern_args(patterns):
    pats = [_as_bytes(p) for p in patterns]
    bufs = [C.create_string_buffer(p, len(p)) if p else None for p in pats]
    ptrs = (C.c_void_p * len(pats))(*[C.cast(b, C.c_void_p) if b is not None else None for b in bufs])
    lens = (C.c_uint32 * len(pats))(*[len(p) for p in pats])
    return pats, bufs, ptrs, lens


class Machine:
    """An oracle machine (with or without failure links)."""

    def __init__(self, patterns, with_failure: bool = True, lib=None):
        self.lib = lib or load()
        self.patterns = [_as_bytes(p) for p in patterns]
        _, self._bufs, ptrs, lens = _pattern_args(self.patterns)
        h = C.c_void_p()
        rc = self.lib.oracle_build(ptrs, lens, len(self.patterns), int(with_failure), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle_build failed ({rc})")
        self.h = h
        self.with_failure = with_failure

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.oracle_free(h)
            self.h = None

    @property
    def num_states(self) -> int:
        return self.lib.oracle_num_states(self.h)

    @property
    def max_len(self) -> int:
        return self.lib.oracle_max_len(self.h)

    def fail(self, s: int) -> int:
        return self.lib.oracle_fail(self.h, s)

    def goto(self, s: int, c) -> int:
        return self.lib.oracle_goto(self.h, s, c if isinstance(c, int) else ord(c))

    def state_of(self, prefix) -> int:
        p = _as_bytes(prefix)
        return self.lib.oracle_state_of(self.h, p, len(p))

    def trace(self, text) -> np.ndarray:
        arr, ptr, n = _text_buf(text)
        out = np.zeros(n, dtype=np.uint32)
        rc = self.lib.oracle_trace(self.h, ptr, n, out.ctypes.data_as(C.POINTER(C.c_uint32)))
        if rc:
            raise ValueError("trace needs the failure-link machine")
        return out

    def _result(self, rc, pairs, M):
        if rc != 0:
            raise MemoryError(f"oracle call failed ({rc})")
        m = int(M.value)
        if m:
            arr = np.ctypeslib.as_array(pairs, shape=(m * 2,)).reshape(m, 2).copy()
        else:
            arr = np.zeros((0, 2), dtype=np.uint32)
        self.lib.oracle_free_buf(C.cast(pairs, C.c_void_p))
        return arr, counts_of(arr, len(self.patterns), self.lib)

    def scan(self, text):
        arr, ptr, n = _text_buf(text)
        pairs, M = C.POINTER(C.c_uint32)(), C.c_uint64()
        rc = self.lib.oracle_scan(self.h, ptr, n, C.byref(pairs), C.byref(M))
        return self._result(rc, pairs, M)

    def scan_mt(self, text, threads: int):
        arr, ptr, n = _text_buf(text)
        pairs, M = C.POINTER(C.c_uint32)(), C.c_uint64()
        rc = self.lib.oracle_scan_mt(self.h, ptr, n, int(threads), C.byref(pairs), C.byref(M))
        return self._result(rc, pairs, M)

    def pfac(self, text):
        arr, ptr, n = _text_buf(text)
        pairs, M = C.POINTER(C.c_uint32)(), C.c_uint64()
        rc = self.lib.oracle_pfac(self.h, ptr, n, C.byref(pairs), C.byref(M))
        return self._result(rc, pairs, M)

    def pfac_walk(self, text, start: int, cap: int = 4096) -> list:
        arr, ptr, n = _text_buf(text)
        out = np.zeros(cap, dtype=np.uint32)
        k = self.lib.oracle_pfac_walk(self.h, ptr, n, start, out.ctypes.data_as(C.POINTER(C.c_uint32)), cap)
        return out[:min(k, cap)].tolist()


def counts_of(matches: np.ndarray, P: int, lib=None) -> np.ndarray:
    lib = lib or load()
    m = np.ascontiguousarray(matches, dtype=np.uint32)
    counts = np.zeros(P, dtype=np.uint64)
    lib.oracle_counts(m.ctypes.data_as(C.POINTER(C.c_uint32)), m.shape[0], P,
                      counts.ctypes.data_as(C.POINTER(C.c_uint64)))
    return counts


def scan(patterns, text, lib=None):
    return Machine(patterns, True, lib).scan(text)


def scan_mt(patterns, text, threads, lib=None):
    return Machine(patterns, True, lib).scan_mt(text, threads)


def pfac(patterns, text, lib=None):
    return Machine(patterns, False, lib).pfac(text)


def brute(patterns, text, lib=None):
    lib = lib or load()
    pats, bufs, ptrs, lens = _pattern_args(patterns)
    arr, ptr, n = _text_buf(text)
    pairs, M = C.POINTER(C.c_uint32)(), C.c_uint64()
    rc = lib.oracle_brute(ptrs, lens, len(pats), ptr, n, C.byref(pairs), C.byref(M))
    if rc != 0:
        raise MemoryError(f"oracle_brute failed ({rc})")
    m = int(M.value)
    res = (np.ctypeslib.as_array(pairs, shape=(m * 2,)).reshape(m, 2).copy() if m
           else np.zeros((0, 2), dtype=np.uint32))
    lib.oracle_free_buf(C.cast(pairs, C.c_void_p))
    return res, counts_of(res, len(pats), lib)
