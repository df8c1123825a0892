"""Python binding of libacgb300 (``include/ac.h``): argument marshalling only.

Every function here has the name of the C entry point it calls. Host buffers
are passed as ``bytes``/``bytearray``/numpy arrays/CPU tensors; device
buffers as CUDA ``torch.Tensor`` objects (PyTorch supplies device memory and
streams). Results come back as numpy arrays: ``matches`` of shape ``(M, 2)``
(uint32 end position, uint32 pattern id, sorted) and ``counts`` (uint64, one
per pattern).

The library is the only implementation: if ``libacgb300.so`` is missing or
cannot be loaded, every call raises — there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libacgb300.so")

AC_OK, AC_EINVAL, AC_ENOMEM, AC_ERANGE, AC_ECUDA, AC_ETIMEDOUT, AC_EAGAIN, AC_EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
AC_U8, AC_PACKED2 = 0, 1
AC_HOST, AC_DEVICE = 0, 1
AC_PLACE_AUTO, AC_PLACE_SMEM, AC_PLACE_HYBRID, AC_PLACE_GLOBAL, AC_PLACE_OPT, AC_PLACE_HYBRID16 = 0, 1, 2, 3, 4, 5
AC_BATCH_NO_COUNTS, AC_BATCH_GRAPH, AC_BATCH_ONE_LAUNCH = 1, 2, 4
AC_MACHINE_DFA, AC_MACHINE_PFAC = 0, 1
AC_KERNEL_AUTO, AC_KERNEL_GENERAL, AC_KERNEL_LEAN, AC_KERNEL_SHORT = 0, 1, 2, 3
AC_BUILDER_HOST, AC_BUILDER_DEVICE = 0, 1
AC_STAGE_DEVICE, AC_STAGE_PINNED = 0, 1

EXPORTED = (
    "ac_build", "ac_free", "ac_save", "ac_load", "ac_stats", "ac_subset", "ac_set_scan_config", "ac_get_scan_config", "ac_tune",
    "ac_scan", "ac_scan_async", "ac_scan_keys_async", "ac_key_shift", "ac_sort_keys_async", "ac_scan_noalloc", "ac_scan_batch", "ac_batch_release", "ac_result_free", "ac_results_take", "ac_serve_create", "ac_serve_submit", "ac_serve_submit_at",
    "ac_serve_poll", "ac_serve_wait", "ac_serve_stats", "ac_serve_destroy", "ac_strerror", "ac_last_error",
    "ac_version", "ac_probe_gather", "ac_probe_launch",
)


class AcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


# ---------------------------------------------------------------- C types
class ac_match(C.Structure):
    _fields_ = [("pos", C.c_uint32), ("pattern_id", C.c_uint32)]


class ac_build_opts(C.Structure):
    _fields_ = [("alphabet", C.c_char_p), ("num_subsets", C.c_uint32), ("placement", C.c_int32),
                ("device", C.c_int32), ("smem_table_bytes", C.c_uint32), ("machine", C.c_int32),
                ("stride", C.c_uint32), ("builder", C.c_uint32)]


class ac_result(C.Structure):
    _fields_ = [("matches", C.POINTER(ac_match)), ("num_matches", C.c_uint64),
                ("counts", C.POINTER(C.c_uint64)), ("num_patterns", C.c_uint32)]


class ac_stats_t(C.Structure):
    _fields_ = [("num_patterns", C.c_uint32), ("num_subsets", C.c_uint32), ("sigma", C.c_uint32),
                ("max_len", C.c_uint32), ("states", C.c_uint64), ("table_bytes", C.c_uint64),
                ("output_entries", C.c_uint64), ("smem_states", C.c_uint64), ("build_ms", C.c_double),
                ("upload_ms", C.c_double), ("device", C.c_int32), ("row_len", C.c_uint32),
                ("threads", C.c_uint32), ("chains", C.c_uint32), ("table2_bytes", C.c_uint64),
                ("scan_placement", C.c_int32), ("scan_stride", C.c_uint32), ("scan_kernel", C.c_int32)]


class ac_subset_view(C.Structure):
    _fields_ = [("id_lo", C.c_uint32), ("id_hi", C.c_uint32), ("max_len", C.c_uint32), ("sigma", C.c_uint32),
                ("states", C.c_uint32), ("smem_states", C.c_uint32), ("table", C.POINTER(C.c_uint32)),
                ("fail", C.POINTER(C.c_uint32)), ("depth", C.POINTER(C.c_uint32)),
                ("out_off", C.POINTER(C.c_uint32)), ("out_ids", C.POINTER(C.c_uint32)),
                ("symbol_of_byte", C.POINTER(C.c_uint8)), ("table2", C.POINTER(C.c_uint32)),
                ("table16", C.POINTER(C.c_uint16)), ("rows16", C.c_uint32),
                ("table_e16", C.POINTER(C.c_uint16)), ("rows_e16", C.c_uint32)]


class ac_scan_config(C.Structure):
    _fields_ = [("row_len", C.c_uint32), ("threads", C.c_uint32), ("chains", C.c_uint32), ("ctas", C.c_uint32),
                ("stage_bytes", C.c_uint32), ("smem_table_bytes", C.c_uint32), ("stride", C.c_uint32),
                ("kernel", C.c_uint32)]


class ac_batch_item(C.Structure):
    _fields_ = [("automaton", C.c_uint32), ("fmt", C.c_int32), ("text", C.c_void_p), ("n", C.c_uint64)]


class ac_serve_opts(C.Structure):
    _fields_ = [("device_mem_budget", C.c_uint64), ("max_batch_items", C.c_uint32), ("max_queue", C.c_uint32),
                ("num_streams", C.c_uint32), ("max_wait_us", C.c_uint32), ("pinned_bytes", C.c_uint64),
                ("staging", C.c_uint32)]


class ac_gather_probe(C.Structure):
    _fields_ = [("ms", C.c_double), ("gathers", C.c_double), ("gathers_per_s", C.c_double),
                ("chains_per_sm", C.c_uint32), ("sms", C.c_uint32)]


class ac_serve_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("launches", C.c_uint64),
                ("items_launched", C.c_uint64), ("queued", C.c_uint64), ("in_flight", C.c_uint64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("mean_batch_items", C.c_double)]


_lock = threading.Lock()
_lib = None


def _declare(lib):
    vp, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int32
    sig = {
        "ac_build": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(u32), u32, C.POINTER(ac_build_opts),
                               C.POINTER(vp)]),
        "ac_free": (None, [vp]),
        "ac_save": (C.c_int, [vp, C.c_char_p]),
        "ac_load": (C.c_int, [C.c_char_p, C.c_int32, C.POINTER(vp)]),
        "ac_stats": (C.c_int, [vp, C.POINTER(ac_stats_t)]),
        "ac_subset": (C.c_int, [vp, u32, C.POINTER(ac_subset_view)]),
        "ac_set_scan_config": (C.c_int, [vp, C.POINTER(ac_scan_config)]),
        "ac_get_scan_config": (C.c_int, [vp, C.POINTER(ac_scan_config)]),
        "ac_tune": (C.c_int, [vp, vp, u64, C.c_int, vp, C.POINTER(ac_scan_config)]),
        "ac_scan": (C.c_int, [vp, vp, u64, C.c_int, C.c_int, vp, C.POINTER(ac_result)]),
        "ac_scan_async": (C.c_int, [vp, vp, u64, C.c_int, vp, vp, u64, vp, vp]),
        "ac_scan_keys_async": (C.c_int, [vp, vp, u64, C.c_int, vp, vp, u64, vp, vp]),
        "ac_key_shift": (C.c_int, [vp]),
        "ac_sort_keys_async": (C.c_int, [vp, u64, vp, vp, u64, vp, vp, vp]),
        "ac_scan_noalloc": (C.c_int, [vp, vp, u64, C.c_int, vp, vp, u64, vp, vp]),
        "ac_scan_batch": (C.c_int, [C.POINTER(vp), u32, C.POINTER(ac_batch_item), u32, C.c_int, u32, vp,
                                    C.POINTER(ac_result)]),
        "ac_batch_release": (None, []),
        "ac_result_free": (None, [C.POINTER(ac_result)]),
        "ac_results_take": (C.c_int, [C.POINTER(ac_result), u32, vp, vp, vp, vp]),
        "ac_serve_create": (C.c_int, [C.POINTER(vp), u32, C.POINTER(ac_serve_opts), C.POINTER(vp)]),
        "ac_serve_submit": (C.c_int, [vp, u32, vp, u64, C.c_int, C.POINTER(u64)]),
        "ac_serve_submit_at": (C.c_int, [vp, u32, vp, u64, C.c_int, u64, C.POINTER(u64)]),
        "ac_serve_poll": (C.c_int, [vp, u64, C.POINTER(ac_result)]),
        "ac_serve_wait": (C.c_int, [vp, u64, u32, C.POINTER(ac_result)]),
        "ac_serve_stats": (C.c_int, [vp, C.POINTER(ac_serve_stats_t)]),
        "ac_serve_destroy": (None, [vp]),
        "ac_strerror": (C.c_char_p, [C.c_int]),
        "ac_last_error": (C.c_char_p, []),
        "ac_version": (C.c_int, []),
        "ac_probe_gather": (C.c_int, [C.c_int, u64, C.c_int, u32, u32, u32, C.POINTER(ac_gather_probe)]),
        "ac_probe_launch": (C.c_int, [C.c_void_p, u32, u32, u32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def lib():
    """The loaded library; raises if it is missing (build it with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise ImportError(f"libacgb300.so is not built ({LIB_PATH}); run __graft_entry__.build()")
                _lib = _declare(C.CDLL(LIB_PATH))
    return _lib


def _check(rc: int, what: str):
    if rc != AC_OK:
        detail = lib().ac_last_error()
        raise AcError(rc, f"{what}: {detail.decode(errors='replace') if detail else ''}")


# ---------------------------------------------------------------- marshalling helpers
def _torch():
    import torch
    return torch


def _is_tensor(x) -> bool:
    t = type(x)
    return t.__module__.startswith("torch") and t.__name__ == "Tensor"


def _stream_ptr(stream):
    if stream is None:
        try:
            torch = _torch()
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _host_bytes(x):
    """(keepalive, pointer, nbytes) for a host buffer."""
    if isinstance(x, (bytes, bytearray, memoryview)):
        arr = np.frombuffer(x, dtype=np.uint8)
    elif _is_tensor(x):
        arr = x.detach().contiguous().view(-1).numpy().view(np.uint8)
    else:
        arr = np.ascontiguousarray(x).view(np.uint8).reshape(-1)
    return arr, C.c_void_p(arr.ctypes.data if arr.size else 0), arr.size


def _device_ptr(t):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("device buffers must be contiguous")
    return C.c_void_p(t.data_ptr())


def _result_to_numpy(r: ac_result, want_counts: bool = True):
    # plain copies out of the library's arrays (no per-size ctypes array types)
    m = int(r.num_matches)
    matches = np.empty((m, 2), dtype=np.uint32)
    if m:
        C.memmove(matches.ctypes.data, r.matches, 8 * m)
    counts = None
    if want_counts:
        P = int(r.num_patterns)
        if P and r.counts:
            counts = np.empty(P, dtype=np.uint64)
            C.memmove(counts.ctypes.data, r.counts, 8 * P)
        else:
            counts = np.zeros(P, dtype=np.uint64)
    lib().ac_result_free(C.byref(r))
    return matches, counts


# numpy view of an ac_result array (field offsets from the ctypes layout)
_RESULT_DTYPE = np.dtype({"names": ["num_matches", "num_patterns"], "formats": [np.uint64, np.uint32],
                          "offsets": [ac_result.num_matches.offset, ac_result.num_patterns.offset],
                          "itemsize": C.sizeof(ac_result)})


def _take_results(outs, n: int, want_counts: bool = True, flat: bool = False):
    """Results outs[0..n) as ``(matches, counts)`` pairs: one copy out of the
    library into two flat arrays (ac_results_take, which releases the
    results), each pair views into them; counts None unless want_counts.
    flat: the arrays themselves, ``(matches, moff, counts, coff)`` -- text i's
    matches are ``matches[moff[i]:moff[i + 1]]`` (and its counts likewise)."""
    if n == 0:
        return (np.zeros((0, 2), np.uint32), np.zeros(1, np.uint64), None, None) if flat else []
    rec = np.frombuffer(outs, dtype=_RESULT_DTYPE, count=n)
    matches = np.empty((int(rec["num_matches"].sum()), 2), dtype=np.uint32)
    moff = np.empty(n + 1, dtype=np.uint64)
    counts = coff = None
    if want_counts:
        counts = np.empty(int(rec["num_patterns"].astype(np.uint64).sum()), dtype=np.uint64)
        coff = np.empty(n + 1, dtype=np.uint64)
    _check(lib().ac_results_take(outs, n, matches.ctypes.data, moff.ctypes.data,
                                 counts.ctypes.data if want_counts else None,
                                 coff.ctypes.data if want_counts else None), "ac_results_take")
    if flat:
        return matches, moff, counts, coff
    mo = moff.tolist()
    ms = [matches[mo[i]:mo[i + 1]] for i in range(n)]
    if not want_counts:
        return [(m, None) for m in ms]
    co = coff.tolist()
    return [(ms[i], counts[co[i]:co[i + 1]]) for i in range(n)]


# ---------------------------------------------------------------- automaton
class Automaton:
    """Owns an ``ac_automaton*``; released by :func:`ac_free` or garbage collection."""

    def __init__(self, handle, num_patterns: int, device: int):
        self.h = handle
        self.num_patterns = num_patterns
        self.device = device

    def __del__(self):
        try:
            ac_free(self)
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.h


def ac_build(patterns, alphabet=None, num_subsets: int = 1, placement: int = AC_PLACE_AUTO,
             device: int = 0, smem_table_bytes: int = 0, machine: int = AC_MACHINE_DFA,
             stride: int = 0, builder: int = AC_BUILDER_HOST) -> Automaton:
    pats = [p.encode() if isinstance(p, str) else bytes(p) for p in patterns]
    # one contiguous buffer; pattern j starts at offs[j] (empty patterns get a NULL pointer)
    blob = np.frombuffer(b"".join(pats) or b"\0", dtype=np.uint8)
    lens_np = np.fromiter((len(p) for p in pats), dtype=np.uint32, count=len(pats))
    offs = np.zeros(len(pats), dtype=np.uint64)
    if len(pats) > 1:
        np.cumsum(lens_np[:-1], out=offs[1:])
    addr = (offs + np.uint64(blob.ctypes.data)).astype(np.uint64)
    addr[lens_np == 0] = 0
    ptrs = addr.ctypes.data_as(C.POINTER(C.c_void_p)) if len(pats) else (C.c_void_p * 1)()
    lens = lens_np.ctypes.data_as(C.POINTER(C.c_uint32)) if len(pats) else (C.c_uint32 * 1)()
    if isinstance(alphabet, str):
        alphabet = alphabet.encode()
    opts = ac_build_opts(alphabet, num_subsets, placement, device, smem_table_bytes, machine, stride, builder)
    h = C.c_void_p()
    _check(lib().ac_build(ptrs, lens, len(pats), C.byref(opts), C.byref(h)), "ac_build")
    del blob, addr, lens_np  # the library copied what it needs
    return Automaton(h, len(pats), device)


def ac_free(a: Automaton):
    if a is not None and a.h:
        lib().ac_free(a.h)
        a.h = None


def ac_save(a: Automaton, path) -> None:
    _check(lib().ac_save(a.h, os.fsencode(path)), "ac_save")


def ac_load(path, device: int = 0) -> Automaton:
    h = C.c_void_p()
    _check(lib().ac_load(os.fsencode(path), device, C.byref(h)), "ac_load")
    st = ac_stats_t()
    _check(lib().ac_stats(h, C.byref(st)), "ac_stats")
    return Automaton(h, int(st.num_patterns), device)


def ac_stats(a: Automaton) -> dict:
    s = ac_stats_t()
    _check(lib().ac_stats(a.h, C.byref(s)), "ac_stats")
    return {f: getattr(s, f) for f, _ in ac_stats_t._fields_}


def ac_subset(a: Automaton, k: int) -> dict:
    v = ac_subset_view()
    _check(lib().ac_subset(a.h, k, C.byref(v)), "ac_subset")
    S, sigma = v.states, v.sigma

    def arr(ptr, n, ty=np.uint32):
        return np.ctypeslib.as_array(ptr, shape=(n,)).astype(ty, copy=True) if n else np.zeros(0, ty)

    out_off = arr(v.out_off, S + 1)
    return {"id_lo": v.id_lo, "id_hi": v.id_hi, "max_len": v.max_len, "sigma": sigma, "states": S,
            "table": arr(v.table, S * sigma).reshape(S, sigma), "fail": arr(v.fail, S), "depth": arr(v.depth, S),
            "out_off": out_off, "out_ids": arr(v.out_ids, int(out_off[-1])),
            "symbol_of_byte": arr(v.symbol_of_byte, 256, np.uint8),
            "table2": arr(v.table2, S * 16).reshape(S, 16) if v.table2 else None,
            "table16": arr(v.table16, v.rows16 * 4, np.uint16).reshape(-1, 4) if v.table16 else None,
            "table_e16": arr(v.table_e16, v.rows_e16 * 4, np.uint16).reshape(-1, 4) if v.table_e16 else None}


def ac_set_scan_config(a: Automaton, row_len: int = 0, threads: int = 0, chains: int = 0, ctas: int = 0,
                       stage_bytes: int = 0, smem_table_bytes: int = 0, stride: int = 0,
                       kernel: int = AC_KERNEL_AUTO):
    cfg = ac_scan_config(row_len, threads, chains, ctas, stage_bytes, smem_table_bytes, stride, kernel)
    _check(lib().ac_set_scan_config(a.h, C.byref(cfg)), "ac_set_scan_config")


def ac_get_scan_config(a: Automaton) -> dict:
    cfg = ac_scan_config()
    _check(lib().ac_get_scan_config(a.h, C.byref(cfg)), "ac_get_scan_config")
    return {f: getattr(cfg, f) for f, _ in ac_scan_config._fields_}


def ac_tune(a: Automaton, d_text, n: int | None = None, fmt: int = AC_U8, stream=None) -> dict:
    cfg = ac_scan_config()
    n = int(d_text.numel() if n is None else n)
    _check(lib().ac_tune(a.h, _device_ptr(d_text), n, fmt, _stream_ptr(stream), C.byref(cfg)), "ac_tune")
    return {f: getattr(cfg, f) for f, _ in ac_scan_config._fields_}


# ---------------------------------------------------------------- scans
def ac_scan(a: Automaton, text, n: int | None = None, fmt: int = AC_U8, stream=None):
    """Scan ``text`` (host buffer or CUDA tensor); returns ``(matches, counts)``."""
    r = ac_result()
    if _is_tensor(text) and text.is_cuda:
        nb = text.numel() * text.element_size()
        nsym = int(n if n is not None else (nb if fmt == AC_U8 else 4 * nb))
        rc = lib().ac_scan(a.h, _device_ptr(text), nsym, fmt, AC_DEVICE, _stream_ptr(stream), C.byref(r))
    else:
        keep, ptr, nb = _host_bytes(text)
        nsym = int(n if n is not None else (nb if fmt == AC_U8 else 4 * nb))
        rc = lib().ac_scan(a.h, ptr, nsym, fmt, AC_HOST, _stream_ptr(stream), C.byref(r))
    _check(rc, "ac_scan")
    return _result_to_numpy(r)


def ac_scan_async(a: Automaton, d_text, n: int, fmt: int, stream, d_matches, cap: int, d_num, d_counts=None):
    """Queue a device-to-device scan: ``d_matches`` (CUDA tensor of >= 2*cap
    int32/uint32 or cap int64), ``d_num`` (CUDA int64 tensor, 1 element),
    ``d_counts`` (CUDA int64 tensor of num_patterns, optional)."""
    rc = lib().ac_scan_async(a.h, _device_ptr(d_text), int(n), fmt, _stream_ptr(stream),
                             _device_ptr(d_matches) if cap else None, int(cap), _device_ptr(d_num),
                             _device_ptr(d_counts) if d_counts is not None else None)
    _check(rc, "ac_scan_async")


def ac_scan_keys_async(a: Automaton, d_text, n: int, fmt: int, stream, d_keys, cap: int, d_num, d_counts=None):
    """Queue the scan up to unsorted keys ``(pos << ac_key_shift(a)) | id`` in
    ``d_keys`` (CUDA int64 tensor of >= cap); count in ``d_num``."""
    rc = lib().ac_scan_keys_async(a.h, _device_ptr(d_text), int(n), fmt, _stream_ptr(stream),
                                  _device_ptr(d_keys) if cap else None, int(cap), _device_ptr(d_num),
                                  _device_ptr(d_counts) if d_counts is not None else None)
    _check(rc, "ac_scan_keys_async")


def ac_key_shift(a: Automaton) -> int:
    return int(lib().ac_key_shift(a.h))


def ac_sort_keys_async(a: Automaton, n: int, d_keys, d_num, cap: int, stream, d_matches, d_num_out):
    rc = lib().ac_sort_keys_async(a.h, int(n), _device_ptr(d_keys) if cap else None, _device_ptr(d_num), int(cap),
                                  _stream_ptr(stream), _device_ptr(d_matches) if cap else None,
                                  _device_ptr(d_num_out))
    _check(rc, "ac_sort_keys_async")


def ac_scan_noalloc(a: Automaton, d_text, n: int, fmt: int, stream, d_matches, cap: int, d_num, d_counts=None):
    """Like :func:`ac_scan_async`, but the library allocates nothing: its
    scratch is a fixed array built into the library (cap <= 262,144; texts
    over 64 KiB must be 16-byte aligned; overlapping calls race)."""
    rc = lib().ac_scan_noalloc(a.h, _device_ptr(d_text), int(n), fmt, _stream_ptr(stream),
                               _device_ptr(d_matches) if cap else None, int(cap), _device_ptr(d_num),
                               _device_ptr(d_counts) if d_counts is not None else None)
    _check(rc, "ac_scan_noalloc")


_ITEM_DTYPE = np.dtype({"names": ["automaton", "fmt", "text", "n"], "formats": [np.uint32, np.int32, np.uint64, np.uint64],
                        "offsets": [ac_batch_item.automaton.offset, ac_batch_item.fmt.offset,
                                    ac_batch_item.text.offset, ac_batch_item.n.offset],
                        "itemsize": C.sizeof(ac_batch_item)})


def ac_scan_batch(automata, items, mem: int = AC_HOST, flags: int = 0, stream=None, flat: bool = False):
    """``items``: list of ``(automaton_index, text, n, fmt)``; texts are host
    buffers (mem=AC_HOST) or CUDA tensors (mem=AC_DEVICE). Returns a list of
    ``(matches, counts)`` (counts None with AC_BATCH_NO_COUNTS), or with
    ``flat=True`` the flat arrays ``(matches, moff, counts, coff)``: item i's
    matches are ``matches[moff[i]:moff[i + 1]]``, its counts
    ``counts[coff[i]:coff[i + 1]]`` (no per-item array objects)."""
    hs = (C.c_void_p * max(1, len(automata)))(*[a.h for a in automata])
    # the item array filled column by column (one ctypes struct per item costs microseconds each)
    arr = np.zeros(max(1, len(items)), dtype=_ITEM_DTYPE)
    keep = []
    if items:
        ai, texts, ns, fmts = zip(*items)
        if mem == AC_DEVICE:
            for t in texts:
                if not t.is_cuda or not t.is_contiguous():
                    raise ValueError("device texts must be contiguous CUDA tensors")
            ptrs = [t.data_ptr() for t in texts]
        else:
            ptrs = []
            for t in texts:
                k, ptr, _ = _host_bytes(t)
                keep.append(k)
                ptrs.append(ptr.value or 0)
        arr["automaton"][:len(items)] = ai
        arr["fmt"][:len(items)] = fmts
        arr["text"][:len(items)] = ptrs
        arr["n"][:len(items)] = ns
    arr_p = arr.ctypes.data_as(C.POINTER(ac_batch_item))
    outs = (ac_result * max(1, len(items)))()
    _check(lib().ac_scan_batch(hs, len(automata), arr_p, len(items), mem, int(flags), _stream_ptr(stream), outs),
           "ac_scan_batch")
    return _take_results(outs, len(items), not (flags & AC_BATCH_NO_COUNTS), flat)


def ac_batch_release():
    lib().ac_batch_release()


# ---------------------------------------------------------------- serving
class Server:
    def __init__(self, handle, automata):
        self.h = handle
        self.automata = automata  # keeps the automata alive for the server's lifetime

    def __del__(self):
        try:
            ac_serve_destroy(self)
        except Exception:
            pass


def ac_serve_create(automata, device_mem_budget: int = 0, max_batch_items: int = 0, max_queue: int = 0,
                    num_streams: int = 0, max_wait_us: int = 0, pinned_bytes: int = 0,
                    staging: int = 0) -> Server:
    hs = (C.c_void_p * max(1, len(automata)))(*[a.h for a in automata])
    opts = ac_serve_opts(device_mem_budget, max_batch_items, max_queue, num_streams, max_wait_us, pinned_bytes,
                         staging)
    h = C.c_void_p()
    _check(lib().ac_serve_create(hs, len(automata), C.byref(opts), C.byref(h)), "ac_serve_create")
    return Server(h, list(automata))


def ac_serve_submit(s: Server, automaton: int, text, n: int | None = None, fmt: int = AC_U8) -> int:
    keep, ptr, nb = _host_bytes(text)
    nsym = int(n if n is not None else (nb if fmt == AC_U8 else 4 * nb))
    t = C.c_uint64()
    _check(lib().ac_serve_submit(s.h, automaton, ptr, nsym, fmt, C.byref(t)), "ac_serve_submit")
    return int(t.value)


def ac_serve_submit_at(s: Server, automaton: int, text, arrival_ns: int, n: int | None = None,
                       fmt: int = AC_U8) -> int:
    """:func:`ac_serve_submit` for a request that arrived at ``arrival_ns``
    (``time.monotonic_ns()`` clock); latency statistics count from then."""
    keep, ptr, nb = _host_bytes(text)
    nsym = int(n if n is not None else (nb if fmt == AC_U8 else 4 * nb))
    t = C.c_uint64()
    _check(lib().ac_serve_submit_at(s.h, automaton, ptr, nsym, fmt, int(arrival_ns), C.byref(t)),
           "ac_serve_submit_at")
    return int(t.value)


def ac_serve_poll(s: Server, ticket: int):
    """``(matches, counts)`` when done, ``None`` while pending."""
    r = ac_result()
    rc = lib().ac_serve_poll(s.h, ticket, C.byref(r))
    if rc == AC_EAGAIN:
        return None
    _check(rc, "ac_serve_poll")
    return _result_to_numpy(r)


def ac_serve_wait(s: Server, ticket: int, timeout_ms: int = 60000):
    r = ac_result()
    _check(lib().ac_serve_wait(s.h, ticket, timeout_ms, C.byref(r)), "ac_serve_wait")
    return _result_to_numpy(r)


def ac_serve_stats(s: Server) -> dict:
    st = ac_serve_stats_t()
    _check(lib().ac_serve_stats(s.h, C.byref(st)), "ac_serve_stats")
    return {f: getattr(st, f) for f, _ in ac_serve_stats_t._fields_}


def ac_serve_destroy(s: Server):
    if s is not None and s.h:
        lib().ac_serve_destroy(s.h)
        s.h = None


def ac_strerror(code: int) -> str:
    return lib().ac_strerror(code).decode()


def ac_last_error() -> str:
    v = lib().ac_last_error()
    return v.decode() if v else ""


def ac_version() -> int:
    return lib().ac_version()


def ac_probe_gather(device: int, table_bytes: int, shared: bool = False, threads: int = 1024, chains: int = 4,
                    steps: int = 1024) -> dict:
    """Dependent random 4-byte lookups per second from a table of
    ``table_bytes`` in global memory (L2 or HBM) or shared memory."""
    out = ac_gather_probe()
    _check(lib().ac_probe_gather(int(device), int(table_bytes), int(bool(shared)), int(threads), int(chains),
                                 int(steps), C.byref(out)), "ac_probe_gather")
    return {f: getattr(out, f) for f, _ in ac_gather_probe._fields_}


def ac_probe_launch(stream=None, launches: int = 1, blocks: int = 1, threads: int = 32) -> None:
    """Enqueue ``launches`` empty kernels on ``stream`` (capturable in a CUDA
    graph): the launch floor of a chain of device operations."""
    _check(lib().ac_probe_launch(_stream_ptr(stream), int(launches), int(blocks), int(threads)), "ac_probe_launch")
