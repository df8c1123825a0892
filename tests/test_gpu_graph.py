"""CUDA-graph capture of the asynchronous scan, as the first call of a
process, and stream order around its overlapped launches.

A caller may capture ac_scan_async into a CUDA graph before it has ever
called it. The library's one-time state (the stream-ordered scratch pool, the
tensor-map encoder, kernel attributes) must then already exist, because a
capture refuses to create it. A child process builds the automata and, with
no scan before, captures one call per case into one graph, replays it twice
and hands the results back; they must equal the oracle's, bit-exact: the
short-text kernel (1 MiB), the lean kernel (a 24 MiB text) and four pattern
subsets (general kernel).
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
THREADS = os.cpu_count() or 4

CHILD = textwrap.dedent("""
    import sys
    import numpy as np, torch
    import workloads
    from paper_1403_1305_gb300 import ac as A
    out = sys.argv[1]
    torch.cuda.set_device(0)
    w1 = workloads.config1()
    w2 = workloads.config1(seed=31, n=24 << 20)
    cases = [(A.ac_build(w1.patterns, alphabet="ACGT"), w1.text),
             (A.ac_build(w2.patterns, alphabet="ACGT"), w2.text),
             (A.ac_build(w1.patterns, alphabet="ACGT", num_subsets=4), w1.text)]
    cap = 1 << 16
    bufs = []
    for a, text in cases:
        bufs.append((a, torch.from_numpy(text).cuda(), text.size,
                     torch.full((2 * cap,), -1, dtype=torch.int32, device="cuda"),
                     torch.zeros(1, dtype=torch.int64, device="cuda"),
                     torch.zeros(a.num_patterns, dtype=torch.int64, device="cuda")))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        cs = torch.cuda.current_stream()
        for a, d, n, d_m, d_num, d_c in bufs:
            A.ac_scan_async(a, d, n, A.AC_U8, cs, d_m, cap, d_num, d_c)
    res = {}
    for rep in range(2):
        g.replay()
        torch.cuda.synchronize()
        for i, (a, d, n, d_m, d_num, d_c) in enumerate(bufs):
            M = int(d_num.item())
            res[f"M{rep}_{i}"] = np.array([M])
            res[f"m{rep}_{i}"] = d_m.view(-1, 2)[:min(M, cap)].cpu().numpy().view(np.uint32)
            res[f"c{rep}_{i}"] = d_c.cpu().numpy()
    np.savez(out, **res)
""")


def test_first_call_captured_in_a_graph(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path / "graph.npz")
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD, out], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = np.load(out)
    w1 = workloads.config1()
    w2 = workloads.config1(seed=31, n=24 << 20)
    for i, (pats, text) in enumerate(((w1.patterns, w1.text), (w2.patterns, w2.text), (w1.patterns, w1.text))):
        wm, wc = oracle.scan_mt(pats, text, THREADS)
        for rep in range(2):
            assert int(res[f"M{rep}_{i}"][0]) == wm.shape[0]
            assert np.array_equal(res[f"m{rep}_{i}"], wm)
            assert np.array_equal(res[f"c{rep}_{i}"], wc)


def test_stream_order_around_overlapped_launches():
    """ac_scan_async's scan and sort may start before the launch ahead of
    them finishes (each waits for it before touching its results), so the
    call must still see the text a kernel just before it wrote, and a kernel
    just after it must see its results. Texts are written into one device
    buffer by a copy kernel right before each call, and the results copied
    out by kernels right after it, all on one stream with no synchronisation
    in between; every call must equal the oracle for the text written
    before it."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_1305_gb300 import ac as A
    torch.cuda.set_device(0)
    rng = np.random.default_rng(77)
    w = workloads.config1()
    a = A.ac_build(w.patterns, alphabet="ACGT")
    texts = [w.text.copy()] + [workloads.embed(rng, w.text, w.patterns, 50 * (i + 1)) for i in range(5)]
    srcs = [torch.from_numpy(t).cuda() for t in texts]
    buf = torch.empty_like(srcs[0])
    cap = 1 << 14
    d_m = torch.empty(2 * cap, dtype=torch.int32, device="cuda")
    d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
    d_c = torch.zeros(a.num_patterns, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    outs = []
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        for rep in range(3):
            for src in srcs:
                buf.copy_(src)
                A.ac_scan_async(a, buf, buf.numel(), A.AC_U8, s, d_m, cap, d_num, d_c)
                outs.append((d_num.clone(), d_m.clone(), d_c.clone()))
    s.synchronize()
    wants = [oracle.scan(w.patterns, t) for t in texts]
    for k, (num, m, c) in enumerate(outs):
        wm, wc = wants[k % len(texts)]
        M = int(num.item())
        assert M == wm.shape[0]
        assert np.array_equal(m.view(-1, 2)[:M].cpu().numpy().view(np.uint32), wm)
        assert np.array_equal(c.cpu().numpy(), wc)
