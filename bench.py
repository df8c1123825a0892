#!/usr/bin/env python
"""Benchmark of the Aho-Corasick scan on GB300.

Workload (default): 256 MiB of i.i.d. uniform DNA text (uint8) against
10,000 distinct patterns of length U[16,64] (half cut from the text), one
machine (K = 1), seeded synthetic data. A step is one pass of the whole hot
path over the text: chunked scan with warm-up, match emission, per-pattern
counts, sort of the matches and conversion to (position, id) records, with
the text resident in HBM (it is larger than L2, so no flush is needed between
steps). The machine is built once beforehand (host time reported apart).

Metric: text GB/s (bytes of text scanned per second, the throughput of the
paper's Eq. (1) with the machine already built). Also reported: the scan
kernel against the HBM roofline, the same metric end to end through the C ABI
with the text in pinned host memory (copy in, scan, results copied out), the
other partitions of the same workload (K = 4/16/64 pattern subsets, 2-bit
packed text), and the oracle on the host cores.

``--impl reference`` times the oracle (plain C Aho-Corasick with failure
links) on the host cores on bounded samples of the same workload.

Multi-GPU (torchrun): every rank scans its own copy (replicas; the scan has
no exchange step), the slowest rank's time counts.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "AC scan text GB/s"
UNIT = "GB/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--subsets", type=int, default=1)
    ap.add_argument("--fmt", default="u8", choices=["u8", "packed2"])
    ap.add_argument("--mib", type=int, default=256, help="text size in MiB")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--no-pfac", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--no-embedded", action="store_true")
    ap.add_argument("--batch-texts", type=int, default=4096)
    ap.add_argument("--serve-requests", type=int, default=200)
    return ap.parse_args()


# ---------------------------------------------------------------- peaks and clocks
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


REASONS = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


class ClockSampler:
    """nvidia-smi samples (every 50 ms) while the warm-up and timed region run."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        cmd = ["nvidia-smi", "-i", str(self.gpu),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "50"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            if self.thread:
                self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(REASONS[1:], parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- distributed plumbing
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, x: float) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- oracle on the host cores
def cpu_baseline(w, target_s: float = 1.5):
    """The oracle (failure-link AC, unchanged) over text chunks on all host
    cores, on a sample of the text sized for ~target_s of wall time."""
    import oracle
    cores = os.cpu_count() or 1
    m = oracle.Machine(w.patterns)
    probe = w.text[: min(w.text.size, 8 << 20)]
    t0 = time.perf_counter()
    m.scan_mt(probe, cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    nbytes = int(min(w.text.size, max(probe.size, probe.size * target_s / dt)))
    sample = w.text[:nbytes]
    t0 = time.perf_counter()
    m.scan_mt(sample, cores)
    dt = time.perf_counter() - t0
    return {"value": nbytes / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {nbytes / 2**20:.0f} MiB of the text, all {len(w.patterns)} patterns, "
                      f"oracle (failure-link Aho-Corasick, C) over {cores} text chunks on {cores} threads",
            "seconds": dt}


def run_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    import oracle
    w = workloads.config2(n=args.mib << 20)
    cores = os.cpu_count() or 1
    m = oracle.Machine(w.patterns)
    sample = min(w.text.size, 32 << 20)
    for i in range(args.warmup):
        m.scan_mt(w.text[:sample], cores)
    t0 = time.perf_counter()
    for i in range(args.steps):
        off = (i * sample) % max(1, w.text.size - sample + 1)
        m.scan_mt(w.text[off:off + sample], cores)
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": w.name, "subsets": 1, "fmt": "u8", "text_bytes": int(w.text.size),
                       "patterns": len(w.patterns)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample >> 20} MiB of the text per step, all patterns, {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def kernel_source_hash():
    """sha256[:16] of the scan kernels' sources (the DRAM traffic of a launch is theirs)."""
    h = hashlib.sha256()
    for name in ("scan_kernel.cuh", "scan_lean.cuh"):
        with open(os.path.join(ROOT, "paper_1403_1305_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_per_launch(workload_key: str, field: str = "dram_bytes"):
    """A per-launch counter of the scan kernel (DRAM bytes, L2 read sectors)
    from a committed ncu summary, if it was taken on the current kernel
    source; else None."""
    path = os.path.join(ROOT, "profiles", "scan_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("kernel_source_sha") != kernel_source_hash():
        return None
    e = d.get("per_launch", {}).get(workload_key)
    return e.get(field) if e else None


def ncu_traffic(workload_key: str):
    return ncu_per_launch(workload_key, "dram_bytes")


def time_device_path(A, torch, a, d_text, n, fmt, steps, warmup, pg, stream, prewarm_s=0.3):
    """Device-resident text: returns (total_s, scan_s_per_step, M).

    Before the `warmup` steps, untimed steps run for `prewarm_s` seconds: on
    a GB300 the first ~50 launches of a process run about 13% slower than
    the steady state (clocks already at their maximum), so a handful of
    warm-up steps alone would time that transient."""
    P = a.num_patterns
    d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
    d_counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    # size the output from one untimed pass
    probe_cap = 1 << 20
    d_keys = torch.empty(probe_cap, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(stream):
        A.ac_scan_keys_async(a, d_text, n, fmt, stream, d_keys, probe_cap, d_num, d_counts)
    stream.synchronize()
    M = int(d_num.item())
    cap = 1 << max(10, int(np.ceil(np.log2(max(M, 1) * 1.25 + 1))))
    d_keys = torch.empty(cap, dtype=torch.int64, device="cuda")
    d_m = torch.empty(cap, dtype=torch.int64, device="cuda")

    def step(ev0=None, ev1=None):
        if ev0 is not None:
            ev0.record(stream)
        A.ac_scan_keys_async(a, d_text, n, fmt, stream, d_keys, cap, d_num, d_counts)
        if ev1 is not None:
            ev1.record(stream)
        A.ac_sort_keys_async(a, n, d_keys, d_num, cap, stream, d_m, d_num)

    t_end = time.perf_counter() + prewarm_s
    while time.perf_counter() < t_end:
        with torch.cuda.stream(stream):
            for _ in range(10):
                step()
        stream.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step()
    stream.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(pg)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        start.record(stream)
        for i in range(steps):
            step(*evs[i])
        end.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    total = start.elapsed_time(end) / 1e3
    scan = sum(e0.elapsed_time(e1) for e0, e1 in evs) / steps / 1e3
    M2 = int(d_num.item())
    assert M2 == M, (M, M2)
    return total, scan, M


def time_async(A, torch, a, d_text, n, fmt, reps, warm=3):
    """Median device time (ms) of ac_scan_async (device in/out) over reps runs."""
    stream = torch.cuda.Stream()
    P = a.num_patterns
    d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
    d_counts = torch.zeros(P, dtype=torch.int64, device="cuda")
    d_keys = torch.empty(1 << 20, dtype=torch.int64, device="cuda")
    with torch.cuda.stream(stream):
        A.ac_scan_keys_async(a, d_text, n, fmt, stream, d_keys, 1 << 20, d_num, d_counts)
    stream.synchronize()
    M = int(d_num.item())
    cap = 1 << max(10, int(np.ceil(np.log2(max(M, 1) * 1.25 + 1))))
    d_m = torch.empty(cap, dtype=torch.int64, device="cuda")
    ts = []
    with torch.cuda.stream(stream):  # untimed steady-state warm-up (see time_device_path)
        t_end = time.perf_counter() + 0.1
        while time.perf_counter() < t_end:
            A.ac_scan_async(a, d_text, n, fmt, stream, d_m, cap, d_num, d_counts)
            stream.synchronize()
    with torch.cuda.stream(stream):
        for i in range(warm + reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            A.ac_scan_async(a, d_text, n, fmt, stream, d_m, cap, d_num, d_counts)
            e1.record(stream)
            e1.synchronize()
            if i >= warm:
                ts.append(e0.elapsed_time(e1))
    return float(np.median(ts)), M, cap, d_m, d_num, d_counts


def bench_lookup_ceilings(A, dev, table_sizes):
    """Dependent random 4-byte lookups per second (ac_probe_gather): a table
    in shared memory (160 KB, the bank-conflict ceiling of one lookup per
    lane), in global memory at the scan tables' sizes (L2-resident when they
    fit) and at 1 GiB (HBM), with 1,024 to 8,192 chains per SM; plus the
    latency of one dependent lookup (one warp, one chain per lane). Each
    random lookup outside shared memory is one 32-byte sector request."""
    out = {"method": "ac_probe_gather: one CTA of 1,024 threads per SM, chains x[j] <- T[hi32(x[j] * words)] + step, "
                     "table of seeded pseudo-random words; CUDA events around one launch after a warm-up launch"}
    sm = A.ac_probe_gather(dev, 160 << 10, shared=True, threads=1024, chains=4, steps=4096)
    out["smem_160KB"] = {"lookups_per_s": sm["gathers_per_s"], "chains_per_sm": sm["chains_per_sm"],
                         "ms": sm["ms"]}
    for name, nbytes in table_sizes:
        rows = []
        for chains in (1, 2, 4, 8):
            r = A.ac_probe_gather(dev, nbytes, shared=False, threads=1024, chains=chains, steps=1024)
            rows.append({"chains_per_sm": r["chains_per_sm"], "lookups_per_s": r["gathers_per_s"]})
        lat = A.ac_probe_gather(dev, nbytes, shared=False, threads=32, chains=1, steps=4096)
        best = max(rows, key=lambda r: r["lookups_per_s"])
        out[name] = {"table_bytes": int(nbytes), "sweep": rows, "best_lookups_per_s": best["lookups_per_s"],
                     "best_chains_per_sm": best["chains_per_sm"],
                     "latency_ns": lat["ms"] * 1e6 / 4096}
    return out


def bench_configs(A, torch, dev, hbm_peak):
    """Config 1 (1 MiB DNA, 100 patterns) and config 3 (64 MiB protein,
    100,000 patterns, table in L2)."""
    out = {}
    w = workloads.config1()
    a = A.ac_build(w.patterns, alphabet="ACGT", device=dev)
    d = torch.from_numpy(w.text).to(f"cuda:{dev}")
    n = w.text.size
    ms, M, cap, d_m, d_num, d_c = time_async(A, torch, a, d, n, A.AC_U8, 20)
    t0 = time.perf_counter()
    for _ in range(20):
        A.ac_scan(a, d)
    wall_ms = (time.perf_counter() - t0) / 20 * 1e3
    # steady state: 100 back-to-back ac_scan_async calls captured in one CUDA graph, replayed
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    graph_ok = True
    try:
        with torch.cuda.graph(g, stream=stream):
            cs = torch.cuda.current_stream()
            for _ in range(100):
                A.ac_scan_async(a, d, n, A.AC_U8, cs, d_m, cap, d_num, d_c)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_ms = e0.elapsed_time(e1) / 1000
        assert int(d_num.item()) == M
    except Exception as ex:  # capture not supported: report it
        graph_ok = False
        graph_ms = None
        out["config1_graph_error"] = str(ex)[:200]
    # the launch floor of that graph: per call, three empty kernels (the
    # call's device operations: zeroing, scan, sort) in the same chain
    floor_ms = None
    try:
        gf = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gf, stream=stream):
            cs = torch.cuda.current_stream()
            for _ in range(100):
                A.ac_probe_launch(cs, 3, 128, 512)
        gf.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            gf.replay()
        e1.record()
        torch.cuda.synchronize()
        floor_ms = e0.elapsed_time(e1) / 1000
    except Exception as ex:
        out["config1_floor_error"] = str(ex)[:200]
    # steady state as one batch of 1000 copies of the text (the default batch
    # path: one text behind separator bytes; matches and counts returned as
    # flat host arrays), wall time of the call
    items = [(0, d, n, A.AC_U8)] * 1000
    A.ac_scan_batch([a], items, mem=A.AC_DEVICE, flat=True)
    A.ac_scan_batch([a], items, mem=A.AC_DEVICE, flat=True)
    t0 = time.perf_counter()
    for _ in range(3):
        A.ac_scan_batch([a], items, mem=A.AC_DEVICE, flat=True)
    batch_ms = (time.perf_counter() - t0) / 3 / 1000 * 1e3
    A.ac_batch_release()
    roof_ms = n / (hbm_peak * 1e9) * 1e3
    out["config1"] = {"workload": w.name, "matches": M, "single_call_device_ms": ms, "single_call_wall_ms": wall_ms,
                      "graph_replayed_ms_per_scan": graph_ms, "batch1000_ms_per_scan": batch_ms,
                      "graph_launch_floor_ms_per_scan": floor_ms,
                      "graph_launch_floor_note": "100 x three empty kernels (128 x 512 threads) in one graph, "
                                                 "the same chain of launches as a call, replayed",
                      "GBps_single": n / ms / 1e6, "GBps_graph": (n / graph_ms / 1e6) if graph_ok else None,
                      "GBps_batch1000": n / batch_ms / 1e6, "roofline_ms": roof_ms,
                      "frac_graph": (roof_ms / graph_ms) if graph_ok else None, "frac_batch1000": roof_ms / batch_ms}
    w = workloads.config3()
    a = A.ac_build(w.patterns, alphabet=w.alphabet, device=dev)
    st = A.ac_stats(a)
    d = torch.from_numpy(w.text).to(f"cuda:{dev}")
    ms, M, *_ = time_async(A, torch, a, d, w.text.size, A.AC_U8, 10)
    # its table (77 MB) is read through L2: the ceiling is random 4-byte reads from a buffer of that size
    probe = max((A.ac_probe_gather(dev, st["table_bytes"], shared=False, threads=1024, chains=c, steps=1024)
                 for c in (2, 4, 8)), key=lambda r: r["gathers_per_s"])
    lk = w.text.size / (ms * 1e-3)
    out["config3"] = {"workload": w.name, "matches": M, "states": st["states"], "table_bytes": st["table_bytes"],
                      "smem_states": st["smem_states"], "median_ms": ms, "GBps": w.text.size / ms / 1e6,
                      "frac_of_hbm": w.text.size / ms / 1e6 / hbm_peak, "build_ms": st["build_ms"],
                      "lookups_per_s": lk, "l2_lookup_ceiling_per_s": probe["gathers_per_s"],
                      "frac_of_l2_lookup_ceiling": lk / probe["gathers_per_s"],
                      "note": "whole scan (ac_scan_async: scan, sort, records) against one dependent lookup per "
                              "symbol at the measured random-read rate of a buffer of the table's size"}
    return out


def bench_pfac(A, torch, dev):
    """The paper's method (failure-less machine, one walk per start position)
    against the failure-folded table, same texts: build (host) and scan."""
    out = {}
    for name, w in (("config1", workloads.config1()), ("config2", workloads.config2()),
                    ("config3", workloads.config3())):
        alph = "ACGT" if w.alphabet == workloads.DNA else w.alphabet
        d = torch.from_numpy(w.text).to(f"cuda:{dev}")
        row = {}
        for kind, mk in (("dfa", A.AC_MACHINE_DFA), ("pfac", A.AC_MACHINE_PFAC)):
            a = A.ac_build(w.patterns, alphabet=alph, device=dev, machine=mk)
            st = A.ac_stats(a)
            ms, M, *_ = time_async(A, torch, a, d, w.text.size, A.AC_U8, 10)
            row[kind] = {"build_ms": st["build_ms"], "scan_ms": ms, "GBps": w.text.size / ms / 1e6, "matches": M,
                         "states": st["states"]}
        row["same_matches"] = row["dfa"]["matches"] == row["pfac"]["matches"]
        out[name] = row
    return out


def bench_paper_shapes(A, torch, dev):
    """The shapes of the paper's Figs. 7-8 (Section V): 70 KB and 100 KB
    inputs against 0.5 M / 1 M / 1.5 M patterns of about 20 bytes (10 / 20 /
    30 MB of patterns). Throughput per Eq. (1): input bytes / total time,
    where the total is machine construction, table upload and the scan with
    results on the host -- the paper's time includes building the machine.
    Both machine kinds, the folded one also built on the GPU
    (AC_BUILDER_DEVICE); synthetic DNA (the paper's data is not
    available). The 7337 B/s of the paper (failure-less machine, 1 thread,
    AMD Opteron, 70 KB, 10 MB of patterns) is context, not a target."""
    rng = np.random.default_rng(1176)
    out = {}
    for P in (500_000, 1_000_000, 1_500_000):
        pats = workloads.random_patterns(rng, P, 15, 25, workloads.DNA)
        mb = sum(len(p) for p in pats) / 1e6
        texts = {kb: workloads.embed(rng, workloads.dna_text(rng, kb * 1000), pats, 50) for kb in (70, 100)}
        rows = {kb: {} for kb in texts}
        for kind, mk, bld in (("dfa", A.AC_MACHINE_DFA, A.AC_BUILDER_HOST),
                              ("dfa_device_build", A.AC_MACHINE_DFA, A.AC_BUILDER_DEVICE),
                              ("pfac", A.AC_MACHINE_PFAC, A.AC_BUILDER_HOST)):
            t0 = time.perf_counter()
            a = A.ac_build(pats, alphabet="ACGT", device=dev, machine=mk, builder=bld)
            build_s = time.perf_counter() - t0
            st = A.ac_stats(a)
            for kb, text in texts.items():
                A.ac_scan(a, text)  # first-call overheads out of the way
                t1 = time.perf_counter()
                m, c = A.ac_scan(a, text)
                scan_s = time.perf_counter() - t1
                rows[kb][kind] = {"eq1_Bps": text.size / (build_s + scan_s), "build_total_ms": build_s * 1e3,
                                  "build_ms": st["build_ms"], "upload_ms": st["upload_ms"], "scan_ms": scan_s * 1e3,
                                  "scan_only_GBps": text.size / scan_s / 1e9, "states": st["states"],
                                  "matches": int(m.shape[0])}
            del a
        for kb in texts:
            rows[kb]["same_matches"] = (rows[kb]["dfa"]["matches"] == rows[kb]["pfac"]["matches"]
                                        == rows[kb]["dfa_device_build"]["matches"])
            out[f"{P // 1000}k_patterns_{mb:.0f}MB_{kb}KB"] = rows[kb]
    return out


def bench_embedded(A, torch, dev):
    """Section V: two texts of the same size, one with patterns embedded and
    one without, should take about the same search time. Timed for the scan
    stage (ac_scan_keys_async: the search, every match emitted as a key, the
    counts) and for the whole path (ac_scan_async: the scan and the sort of
    the matches into records, work that grows with the number of matches)."""
    w = workloads.config2(n=64 << 20)
    a = A.ac_build(w.patterns, alphabet="ACGT", device=dev)
    rng = np.random.default_rng(1177)
    plain = w.text
    rich = workloads.embed(rng, plain, w.patterns, 100_000)
    res = {}
    stream = torch.cuda.Stream()
    for name, t in (("plain", plain), ("embedded_100k", rich)):
        d = torch.from_numpy(t).to(f"cuda:{dev}")
        ms, M, *_ = time_async(A, torch, a, d, t.size, A.AC_U8, 10)
        _, scan_s, _ = time_device_path(A, torch, a, d, t.size, A.AC_U8, 10, 3, None, stream, prewarm_s=0.1)
        res[name] = {"scan_ms": scan_s * 1e3, "scan_and_sort_ms": ms, "matches": M}
    res["time_ratio"] = res["embedded_100k"]["scan_ms"] / res["plain"]["scan_ms"]
    res["time_ratio_with_sort"] = res["embedded_100k"]["scan_and_sort_ms"] / res["plain"]["scan_and_sort_ms"]
    res["note"] = ("time_ratio: scan stage (the search); time_ratio_with_sort: with the sort of the matches into "
                   "records (radix sort of ~131k keys against a rank sort of ~5k)")
    return res


def bench_batch(A, torch, dev, args):
    """4,096 DNA texts (log-uniform 1 KiB..4 MiB) against 8 resident pattern
    sets: one ac_scan_batch -- texts one automaton at a time as one text (the
    default for byte texts), and the one-launch arena with its kept plan
    replayed as a CUDA graph -- against one ac_scan_async call per text,
    texts resident on the device in all."""
    w = workloads.config4(num_texts=args.batch_texts)
    autos = [A.ac_build(s, alphabet="ACGT", device=dev) for s in w.pattern_sets]
    d_texts = [torch.from_numpy(t).to(f"cuda:{dev}") for t in w.texts]
    total = int(sum(t.size for t in w.texts))
    items = [(int(a), d, t.size, A.AC_U8) for a, d, t in zip(w.set_of_text, d_texts, w.texts)]
    torch.cuda.synchronize()
    # plan + autotune, then timed graph replays (results copied to the host and split per text)
    fl = A.AC_BATCH_GRAPH | A.AC_BATCH_NO_COUNTS
    t0 = time.perf_counter()
    res = A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=fl)
    plan_s = time.perf_counter() - t0
    A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=fl)
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        res = A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=fl)
    batched_s = (time.perf_counter() - t0) / reps
    M = sum(m.shape[0] for m, _ in res)
    # the default path for byte texts: one text per automaton; the matches
    # come back as one flat array with per-text offsets
    fs = A.AC_BATCH_NO_COUNTS
    res_s = A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=fs, flat=True)
    t0 = time.perf_counter()
    for _ in range(reps):
        res_s = A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=fs, flat=True)
    segments_s = (time.perf_counter() - t0) / reps
    M_s = int(res_s[0].shape[0])
    # the same with one (matches, counts) pair of array views per text
    A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=fs)
    t0 = time.perf_counter()
    for _ in range(reps):
        A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=fs)
    segments_views_s = (time.perf_counter() - t0) / reps
    # the same with per-text dense count arrays copied to the host as well
    A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=A.AC_BATCH_GRAPH)
    t0 = time.perf_counter()
    A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=A.AC_BATCH_GRAPH)
    counts_s = time.perf_counter() - t0
    # one launch sequence per text: ac_scan_async on one stream, one sync at the end
    stream = torch.cuda.Stream()
    caps = [max(4096, t.size // 512) for t in w.texts]
    d_m = torch.empty(max(caps), dtype=torch.int64, device=f"cuda:{dev}")
    d_num = torch.zeros(len(items), dtype=torch.int64, device=f"cuda:{dev}")
    d_c = torch.empty(max(a.num_patterns for a in autos), dtype=torch.int64, device=f"cuda:{dev}")

    def per_call():
        with torch.cuda.stream(stream):
            for i, (ai, d, n, f) in enumerate(items):
                A.ac_scan_async(autos[ai], d, n, f, stream, d_m, caps[i], d_num[i:i + 1], d_c[:autos[ai].num_patterns])
        stream.synchronize()

    per_call()
    t0 = time.perf_counter()
    per_call()
    per_call_s = time.perf_counter() - t0
    M_calls = int(d_num.sum().item())
    A.ac_batch_release()
    best_s = min(segments_s, batched_s)
    return {"workload": w.name, "texts": len(items), "text_bytes": total, "pattern_sets": w.meta["set_sizes"],
            "batched_GBps": total / best_s / 1e9, "batched_ms": best_s * 1e3,
            "per_call_GBps": total / per_call_s / 1e9, "per_call_ms": per_call_s * 1e3,
            "speedup": per_call_s / best_s,
            "one_text_per_automaton_ms": segments_s * 1e3, "one_launch_graph_ms": batched_s * 1e3,
            "one_text_per_automaton_views_per_text_ms": segments_views_s * 1e3,
            "plan_and_autotune_ms": plan_s * 1e3,
            "one_launch_graph_with_counts_ms": counts_s * 1e3,
            "count_array_bytes": int(sum(autos[int(a)].num_patterns for a in w.set_of_text) * 8),
            "matches": M, "matches_one_text_per_automaton": M_s, "matches_per_call_path": M_calls,
            "batched_path": ("ac_scan_batch(AC_DEVICE, AC_BATCH_NO_COUNTS, flat=True): texts gathered one "
                             "automaton at a time into one text behind separator bytes, one single-text scan + sort "
                             "each, matches to the host as one array with per-text offsets") if segments_s <= batched_s else
                            ("ac_scan_batch(AC_DEVICE, AC_BATCH_GRAPH|AC_BATCH_NO_COUNTS): arena copy + 1 "
                             "persistent scan + sort + records, matches to the host per text"),
            "per_call_path": "ac_scan_async per text (device results), one stream"}


def bench_serve(A, torch, dev, args):
    """16 resident automata (8 DNA x 5,000, 8 protein x 20,000 patterns);
    Poisson arrivals of texts with log-uniform lengths in [4 KiB, 64 MiB];
    rate raised x1.5 until throughput stops growing. Continuous batching
    server against one synchronous ac_scan per request in arrival order.
    Latency counts from each request's scheduled arrival in both arms (the
    server is told it through ac_serve_submit_at), so queueing before the
    server, or behind earlier requests in the per-request arm, is counted.
    Request texts sit in page-locked host memory in both arms. Reported at
    the rate of the best served throughput (median of three runs each) and
    at the highest rate the server keeps up with (arrivals completed at
    >= 85% of the offered rate)."""
    w = workloads.config5_sets()
    autos = [A.ac_build(s, alphabet=a, device=dev) for s, a in zip(w.pattern_sets, w.set_alphabet)]
    rng = np.random.default_rng(1055)
    # one 64 MiB text per alphabet kind, page-locked; a protein set's text maps
    # Zipf ranks through that set's letter order (same law as drawing it directly)
    def pinned(x):
        return torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy()
    dna_pool = pinned(workloads.dna_text(rng, 64 << 20))
    ranks = None
    pools = []
    for letters, probs in w.set_letters:
        if probs is None:
            pools.append(dna_pool)
            continue
        if ranks is None:
            ranks = workloads.iid_text(rng, 64 << 20, np.arange(len(letters), dtype=np.uint8), probs)
        pools.append(pinned(np.asarray(letters, dtype=np.uint8)[ranks]))

    def make(count, rate):
        t, sets, lens = workloads.request_stream(rng, rate, count)
        reqs = []
        for ti, si, L in zip(t, sets, lens):
            pool = pools[int(si)]
            o = int(rng.integers(0, pool.size - int(L) + 1))
            reqs.append((float(ti), int(si), pool[o:o + int(L)]))
        return reqs

    def run_server(reqs, staging=A.AC_STAGE_DEVICE):
        srv = A.ac_serve_create(autos, num_streams=3, max_batch_items=64, max_wait_us=100,
                                device_mem_budget=8 << 30, staging=staging)
        tickets = [None] * len(reqs)
        start = time.perf_counter()
        start_ns = time.monotonic_ns()

        # several producer threads share the arrival stream; each request is
        # submitted at (or, when a producer lags, after) its scheduled time and
        # carries that time as its arrival
        nprod = 4
        ths = []
        for k in range(nprod):
            def prod(k=k):
                for i in range(k, len(reqs), nprod):
                    ta, si, txt = reqs[i]
                    d = start + ta - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    tickets[i] = A.ac_serve_submit_at(srv, si, txt, start_ns + int(ta * 1e9))
            ths.append(threading.Thread(target=prod))
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        for tk in tickets:
            A.ac_serve_wait(srv, tk, 600_000)
        end = time.perf_counter()
        st = A.ac_serve_stats(srv)
        A.ac_serve_destroy(srv)
        return end - start, st

    def run_per_request(reqs):
        lat = []
        start = time.perf_counter()
        for ta, si, txt in reqs:
            d = start + ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            A.ac_scan(autos[si], txt)
            lat.append((time.perf_counter() - start - ta) * 1e3)
        return time.perf_counter() - start, lat

    # raise the offered rate x1.5 until throughput stops growing (no gain of
    # 3% over the best for three rates in a row): past the point where the
    # server keeps up with arrivals, queued requests coalesce into larger
    # batches and throughput still grows
    sweep, rate, best, flat = [], 50.0, 0.0, 0
    for _ in range(24):
        reqs = make(args.serve_requests, rate)
        nbytes = sum(r[2].size for r in reqs)
        el, st = run_server(reqs)
        thr = nbytes / el / 1e9
        offered = len(reqs) / max(reqs[-1][0], 1e-9)
        sweep.append({"rate_hz": rate, "GBps": thr, "req_per_s": len(reqs) / el, "offered_req_per_s": offered,
                      "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_batch_items": st["mean_batch_items"],
                      "launches": st["launches"], "kept_up": len(reqs) / el >= 0.85 * offered})
        flat = flat + 1 if thr < 1.03 * best else 0
        best = max(best, thr)
        if flat >= 3:
            break
        rate *= 1.5
    top = max(sweep, key=lambda r: r["GBps"])
    # the same requests at that rate: served (texts staged in device memory,
    # then in the pinned slab) and one ac_scan per request
    reqs = make(args.serve_requests, top["rate_hz"])
    nbytes = sum(r[2].size for r in reqs)
    # three runs of each path, the median by elapsed time
    el_d, st_d = sorted((run_server(reqs) for _ in range(3)), key=lambda x: x[0])[1]
    el_p, st_p = sorted((run_server(reqs, A.AC_STAGE_PINNED) for _ in range(3)), key=lambda x: x[0])[1]
    el, lat = sorted((run_per_request(reqs) for _ in range(3)), key=lambda x: x[0])[1]
    served = nbytes / el_d / 1e9
    per_req = nbytes / el / 1e9
    kept = [r for r in sweep if r["kept_up"]]
    at_kept = None
    if kept:
        # both arms at the highest rate the server keeps up with
        reqs_k = make(args.serve_requests, kept[-1]["rate_hz"])
        nb_k = sum(r[2].size for r in reqs_k)
        el_k, st_k = run_server(reqs_k)
        el_kr, lat_k = run_per_request(reqs_k)
        at_kept = {"rate_hz": kept[-1]["rate_hz"], "offered_req_per_s": len(reqs_k) / max(reqs_k[-1][0], 1e-9),
                   "served_GBps": nb_k / el_k / 1e9, "served_req_per_s": len(reqs_k) / el_k,
                   "served_p50_ms": st_k["p50_ms"], "served_p99_ms": st_k["p99_ms"],
                   "per_request_GBps": nb_k / el_kr / 1e9, "per_request_req_per_s": len(reqs_k) / el_kr,
                   "per_request_p50_ms": float(np.percentile(lat_k, 50)),
                   "per_request_p99_ms": float(np.percentile(lat_k, 99)),
                   "speedup": el_kr / el_k}
    return {"workload": w.name, "requests_per_rate": args.serve_requests,
            "rate_hz_at_best": top["rate_hz"], "bytes_at_best": nbytes,
            "served_GBps": served, "served_p50_ms": st_d["p50_ms"], "served_p99_ms": st_d["p99_ms"],
            "served_mean_batch_items": st_d["mean_batch_items"],
            "served_pinned_staging_GBps": nbytes / el_p / 1e9, "served_pinned_staging_p50_ms": st_p["p50_ms"],
            "per_request_GBps": per_req, "per_request_p50_ms": float(np.percentile(lat, 50)),
            "per_request_p99_ms": float(np.percentile(lat, 99)),
            "speedup": served / per_req, "at_highest_rate_kept_up": at_kept,
            "latency": "from each request's scheduled arrival to its result on the host, both arms",
            "served_path": "ac_serve_* (3 streams, <=64 requests per launch, page-locked host texts copied into "
                           "device memory by ac_serve_submit_at; 4 producer threads)",
            "per_request_path": "ac_scan(page-locked host text) per request in arrival order",
            "sweep": sweep}


def _r(x, nd=3):
    """x rounded to nd significant digits (None stays None)."""
    if x is None or not isinstance(x, (int, float)):
        return x
    return float(f"{x:.{nd}g}")


def summary(line):
    """The figures of every section in a few hundred bytes, printed as the
    line's last key so that a reader keeping only the end of the output
    still has them."""
    g = line.get
    out = {"value_GBps": _r(g("value")), "scan_kernel_ms": _r(g("roofline", {}).get("kernel_ms")),
           "frac_of_hbm": _r(g("roofline", {}).get("frac")), "e2e_GBps": _r((g("e2e") or {}).get("value"))}
    lc = g("lookup_ceilings") or {}
    if lc:
        out["ceilings_G_lookups_per_s"] = {"smem": _r(lc["smem_160KB"]["lookups_per_s"] / 1e9),
                                           "l2_table": _r(lc["table"]["best_lookups_per_s"] / 1e9),
                                           "hbm": _r(lc["hbm_1GiB"]["best_lookups_per_s"] / 1e9)}
    if g("variants"):
        out["variants_scan_ms"] = {k: _r(v["scan_ms"]) for k, v in g("variants").items()}
    c = g("configs") or {}
    if "config1" in c:
        c1 = c["config1"]
        out["config1_us"] = {"one_call": _r(c1["single_call_device_ms"] * 1e3),
                             "graph": _r((c1["graph_replayed_ms_per_scan"] or 0) * 1e3),
                             "batch1000": _r(c1["batch1000_ms_per_scan"] * 1e3),
                             "graph_launch_floor": _r((c1.get("graph_launch_floor_ms_per_scan") or 0) * 1e3)}
    if "config3" in c:
        out["config3"] = {"ms": _r(c["config3"]["median_ms"]), "frac_l2": _r(c["config3"]["frac_of_l2_lookup_ceiling"])}
    if g("pfac"):
        out["pfac_scan_ms_dfa_vs_failureless"] = {k: [_r(v["dfa"]["scan_ms"]), _r(v["pfac"]["scan_ms"])]
                                                  for k, v in g("pfac").items()}
    if g("paper_shapes"):
        out["paper_eq1_kBps"] = {k: {kk: _r(vv["eq1_Bps"] / 1e3) for kk, vv in v.items() if isinstance(vv, dict)}
                                 for k, v in g("paper_shapes").items() if k.endswith("70KB")}
    if g("embedded_check"):
        out["embedded_time_ratio"] = {"scan": _r(g("embedded_check")["time_ratio"]),
                                      "with_sort": _r(g("embedded_check")["time_ratio_with_sort"])}
    b = g("batch")
    if b:
        out["batch"] = {"batched_GBps": _r(b["batched_GBps"]), "per_call_GBps": _r(b["per_call_GBps"]),
                        "speedup": _r(b["speedup"])}
    sv = g("serve")
    if sv:
        out["serve"] = {k: _r(sv.get(k)) for k in ("served_GBps", "per_request_GBps", "speedup", "served_p50_ms",
                                                   "served_p99_ms", "per_request_p50_ms", "per_request_p99_ms")}
        k = sv.get("at_highest_rate_kept_up")
        if k:
            out["serve_kept_up"] = {kk: _r(k[kk]) for kk in ("rate_hz", "served_GBps", "per_request_GBps", "speedup",
                                                             "served_p50_ms", "served_p99_ms", "per_request_p50_ms",
                                                             "per_request_p99_ms")}
    cb = g("cpu_baseline")
    if cb:
        out["cpu_baseline_GBps"] = _r(cb["value"])
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_1403_1305_gb300 import ac as A

    world, rank, local, pg = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()
    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    w = workloads.config2(n=args.mib << 20)
    fmt = A.AC_U8 if args.fmt == "u8" else A.AC_PACKED2
    host_text = w.text if fmt == A.AC_U8 else workloads.pack2(w.text)
    n = int(w.text.size)
    nbytes = int(host_text.size)
    t0 = time.perf_counter()
    a = A.ac_build(w.patterns, alphabet="ACGT", num_subsets=args.subsets, device=dev)
    build_s = time.perf_counter() - t0
    st = A.ac_stats(a)
    d_text = torch.from_numpy(host_text).to(f"cuda:{dev}")
    stream = torch.cuda.Stream()

    with ClockSampler(dev) as clk:
        total, scan_s, M = time_device_path(A, torch, a, d_text, n, fmt, args.steps, args.warmup, pg, stream)
    total = max_over_ranks(pg, total)
    value = nbytes * world * args.steps / total / 1e9
    clocks = clk.summary()

    # roofline of the scan kernel: the text read once from HBM (bound), against
    # K lookups per symbol at 32 shared-memory lookups per clock per SM
    achieved = nbytes / scan_s / 1e9
    lookups = args.subsets * n
    lookup_rate_peak = n_sm * 32 * sm_mhz * 1e6
    t_hbm = nbytes / (hbm_peak * 1e9)
    t_lookup = lookups / lookup_rate_peak
    bound = "hbm" if t_hbm >= t_lookup else "smem_lookup"
    key = f"{w.name}-K{args.subsets}-{args.fmt}"
    roofline = {"bound": bound, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": ncu_traffic(key),
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "kernel": ("lean_kernel" if st["scan_kernel"] == A.AC_KERNEL_LEAN else "scan_kernel")
                          + " (+ memsets, error mark)", "kernel_ms": scan_s * 1e3,
                "algorithmic_bytes_per_launch": nbytes,
                "roofline_ms": max(t_hbm, t_lookup) * 1e3,
                "frac_of_roofline_time": max(t_hbm, t_lookup) / scan_s,
                "lookup_peak_per_s": lookup_rate_peak, "lookups_per_launch": lookups}
    # the ceilings the lookups meet, measured on this device: random 4-byte
    # lookups in shared memory (bank conflicts), in L2 at this table's size,
    # and in HBM
    ceilings = bench_lookup_ceilings(A, dev, [("table", st["table_bytes"]), ("hbm_1GiB", 1 << 30)])
    l2_ceiling = ceilings["table"]["best_lookups_per_s"]
    smem_ceiling = ceilings["smem_160KB"]["lookups_per_s"]
    roofline["lookups_per_s"] = lookups / scan_s
    roofline["frac_of_measured_smem_lookup_ceiling"] = lookups / scan_s / smem_ceiling
    # the bound that holds in practice: L2 read requests (table rows beyond
    # shared memory, text stages), per launch from the ncu summary, over the
    # live kernel time, against the measured ceiling of random 32-byte L2
    # reads at this table's size
    sectors = ncu_per_launch(key, "l2_read_sectors")
    if sectors:
        roofline["l2_requests"] = {"sectors_per_launch": sectors,
                                   "achieved_gsectors_per_s": sectors / scan_s / 1e9,
                                   "ceiling_gsectors_per_s": l2_ceiling / 1e9,
                                   "frac": sectors / scan_s / l2_ceiling,
                                   "ceiling_source": "ac_probe_gather: random 4-byte reads (one 32-byte sector "
                                                     "each) over a buffer of the table's size, this device"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": w.name, "text_bytes": nbytes, "symbols": n, "fmt": args.fmt,
                       "patterns": len(w.patterns), "pattern_len": [16, 64], "subsets": args.subsets,
                       "states": st["states"], "table_bytes": st["table_bytes"], "smem_states": st["smem_states"],
                       "matches": M, "build_ms": build_s * 1e3, "parallelism": f"replicas{world}",
                       "l2": (f"text ({nbytes / 2**20:.0f} MiB) larger than L2 (129 MB): no flush between steps"
                              if nbytes > 129e6 else f"text ({nbytes / 2**20:.0f} MiB) fits in L2: a warm-L2 figure"),
                       "scan_config": A.ac_get_scan_config(a),
                       "scan_placement": {0: "auto", 1: "smem", 2: "hybrid", 3: "global", 4: "optimistic prefix",
                                          5: "16-bit prefix"}.get(st["scan_placement"], str(st["scan_placement"])),
                       "symbols_per_lookup": st["scan_stride"],
                       "scan_kernel": {1: "general", 2: "lean", 3: "short"}.get(st["scan_kernel"], str(st["scan_kernel"]))},
            "roofline": roofline, "lookup_ceilings": ceilings, "clocks": clocks,
            "gpu_launches": 4 * args.steps,
            "gpu_launches_note": "own kernels per step: zeroing of the counter, error word and counts; scan; "
                                 "error mark; rank sort + record conversion"}

    if not args.no_e2e:
        # end to end through the C ABI: pinned host text in, host results out
        pinned = torch.from_numpy(host_text).pin_memory()
        for _ in range(2):
            A.ac_scan(a, pinned, n=n, fmt=fmt)
        barrier(pg)
        times = []
        for _ in range(max(3, args.steps // 4)):
            t0 = time.perf_counter()
            m, c = A.ac_scan(a, pinned, n=n, fmt=fmt)
            times.append(time.perf_counter() - t0)
        e2e_s = max_over_ranks(pg, statistics.median(times))
        line["e2e"] = {"value": nbytes * world / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": int(m.shape[0] * 8 + c.size * 8 + 16),
                       "api": "ac_scan(host pinned text) -> host matches + counts", "ms": e2e_s * 1e3}

    if not args.no_variants:
        var = {}
        for K, f in ((4, "u8"), (16, "u8"), (64, "u8"), (1, "packed2"), (16, "packed2")):
            if K == args.subsets and f == args.fmt:
                continue
            fm = A.AC_U8 if f == "u8" else A.AC_PACKED2
            ht = w.text if fm == A.AC_U8 else workloads.pack2(w.text)
            av = A.ac_build(w.patterns, alphabet="ACGT", num_subsets=K, device=dev)
            dt = torch.from_numpy(ht).to(f"cuda:{dev}")
            tt, ss, mm = time_device_path(A, torch, av, dt, n, fm, max(3, args.steps // 4), 2, pg, stream,
                                          prewarm_s=0.1)
            lk = K * n / max(1, A.ac_stats(av)["scan_stride"])  # dependent lookups per launch
            steps_v = max(3, args.steps // 4)
            var[f"K{K}-{f}"] = {"GBps": ht.size * steps_v / tt / 1e9, "symbols_per_s": n * steps_v / tt,
                                "scan_ms": ss * 1e3, "matches": mm, "lookups_per_s": lk / ss,
                                "symbols_per_lookup": A.ac_stats(av)["scan_stride"],
                                "frac_of_nominal_smem_lookup_peak": lk / ss / lookup_rate_peak,
                                "frac_of_measured_smem_lookup_ceiling": lk / ss / smem_ceiling,
                                "smem_states": A.ac_stats(av)["smem_states"], "states": A.ac_stats(av)["states"]}
            del av, dt
        line["variants"] = var

    if rank == 0 and not args.no_configs:
        line["configs"] = bench_configs(A, torch, dev, hbm_peak)
    if rank == 0 and not args.no_pfac:
        line["pfac"] = bench_pfac(A, torch, dev)
    if rank == 0 and not args.no_paper:
        line["paper_shapes"] = bench_paper_shapes(A, torch, dev)
    if rank == 0 and not args.no_embedded:
        line["embedded_check"] = bench_embedded(A, torch, dev)
    if rank == 0 and not args.no_batch:
        line["batch"] = bench_batch(A, torch, dev, args)
    if rank == 0 and not args.no_serve:
        line["serve"] = bench_serve(A, torch, dev, args)

    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w)

    if rank == 0:
        line["summary"] = summary(line)  # last key: a short digest of every section
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
