"""ac_scan_noalloc: the scan for callers that must not allocate device memory.

Such callers (a process whose device memory another allocator reserved in
advance, a latency-critical loop that cannot take an allocation's implicit
synchronisation) get an entry point whose scratch is a fixed array compiled
into the library. These tests call it through the C ABI and check that two
calls in a row give exactly what the ordinary asynchronous entry point gives,
so the shared array is cleared properly between calls. This file sorts last
so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import workloads
from paper_1403_1305_gb300 import ac as A

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def run(fn, a, d_text, n, cap, fmt=A.AC_U8):
    d_m = torch.zeros(2 * max(cap, 1), dtype=torch.int32, device="cuda")
    d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
    d_c = torch.zeros(a.num_patterns, dtype=torch.int64, device="cuda")
    fn(a, d_text, n, fmt, None, d_m, cap, d_num, d_c)
    torch.cuda.synchronize()
    M = int(d_num.item())
    m = d_m.view(-1, 2)[:min(M, cap)].cpu().numpy().view(np.uint32)
    return M, m, d_c.cpu().numpy()


def test_two_calls_in_a_row_match_the_allocating_entry_point():
    w1 = workloads.config1()
    w2 = workloads.config1(seed=77, n=300_001)
    a1 = A.ac_build(w1.patterns, alphabet="ACGT")
    a2 = A.ac_build(w2.patterns, alphabet="ACGT")
    cases = [(a1, torch.from_numpy(w1.text).cuda(), w1.text.size),
             (a2, torch.from_numpy(w2.text).cuda(), w2.text.size)]
    cap = 8192
    for a, d, n in cases + cases:          # each input twice, alternating
        want = run(A.ac_scan_async, a, d, n, cap)
        got = run(A.ac_scan_noalloc, a, d, n, cap)
        assert want[0] > 0
        assert got[0] == want[0]
        assert np.array_equal(got[1], want[1])
        assert np.array_equal(got[2], want[2])


def test_short_unaligned_and_packed_texts():
    rng = np.random.default_rng(5)
    text = workloads.dna_text(rng, 40_000)
    pats = workloads.draw_patterns(rng, text, 50, 4, 12, 0.6, np.frombuffer(b"ACGT", np.uint8))
    a = A.ac_build(pats, alphabet="ACGT")
    buf = torch.zeros(text.size + 16, dtype=torch.uint8, device="cuda")
    for off, n in ((3, 40_000), (0, 17), (5, 33)):
        view = buf[off:off + n]
        view.copy_(torch.from_numpy(text[:n]).cuda())
        want = run(A.ac_scan_async, a, view, n, 4096)
        got = run(A.ac_scan_noalloc, a, view, n, 4096)
        assert got[0] == want[0] and np.array_equal(got[1], want[1]) and np.array_equal(got[2], want[2])
    packed = torch.from_numpy(workloads.pack2(text)).cuda()
    want = run(A.ac_scan_async, a, packed, text.size, 4096, A.AC_PACKED2)
    got = run(A.ac_scan_noalloc, a, packed, text.size, 4096, A.AC_PACKED2)
    assert got[0] == want[0] and np.array_equal(got[1], want[1])


def test_capacity_beyond_the_fixed_limit_is_refused():
    a = A.ac_build([b"ACGT"], alphabet="ACGT")
    d = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(A.AcError) as e:
        run(A.ac_scan_noalloc, a, d, 64, (1 << 18) + 1)
    assert e.value.code == A.AC_ERANGE


def test_empty_text_and_zero_capacity():
    """n = 0 (the set-up call a caller makes at initialisation) and cap = 0
    (count only): the counter and the counts come back right although the
    shared array still holds the previous call's contents."""
    w = workloads.config1()
    a = A.ac_build(w.patterns, alphabet="ACGT")
    d = torch.from_numpy(w.text).cuda()
    M, _, c = run(A.ac_scan_noalloc, a, d, w.text.size, 8192)      # leaves matches in the array
    assert M > 0
    d_num = torch.full((1,), 12345, dtype=torch.int64, device="cuda")
    d_c = torch.full((a.num_patterns,), 7, dtype=torch.int64, device="cuda")
    A.ac_scan_noalloc(a, d, 0, A.AC_U8, None, None, 0, d_num, d_c)
    torch.cuda.synchronize()
    assert int(d_num.item()) == 0 and int(d_c.abs().sum().item()) == 0
    A.ac_scan_noalloc(a, d, w.text.size, A.AC_U8, None, None, 0, d_num, d_c)
    torch.cuda.synchronize()
    assert int(d_num.item()) == M and np.array_equal(d_c.cpu().numpy(), c)


CHILD = r'''
import hashlib, json, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import workloads
from paper_1403_1305_gb300 import ac as A
torch.cuda.set_device(0)
w = workloads.config1()
a = A.ac_build(w.patterns, alphabet="ACGT")   # tables from cudaMalloc, not the scratch allocator
d = torch.from_numpy(w.text).cuda()
d_m = torch.zeros(2 * 8192, dtype=torch.int32, device="cuda")
d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
d_c = torch.zeros(a.num_patterns, dtype=torch.int64, device="cuda")
out = {{}}
try:
    A.ac_scan_async(a, d, w.text.size, A.AC_U8, None, d_m, 8192, d_num, d_c)
    out["async"] = 0
except A.AcError as e:
    out["async"] = e.code
for k in range(2):
    A.ac_scan_noalloc(a, d, w.text.size, A.AC_U8, None, d_m, 8192, d_num, d_c)
    torch.cuda.synchronize()
    M = int(d_num.item())
    h = hashlib.sha256(d_m.view(-1, 2)[:M].cpu().numpy().tobytes() + d_c.cpu().numpy().tobytes()).hexdigest()
    out["noalloc%d" % k] = [M, h]
print(json.dumps(out))
'''


def test_allocates_nothing():
    """With every scratch allocation of the library made to fail
    (AC_FAULT_ALLOC=0), ac_scan_async reports AC_ENOMEM while
    ac_scan_noalloc still scans, twice, to the same result as an
    unrestricted run."""
    import hashlib
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env["AC_FAULT_ALLOC"] = "0"
    env.pop("AC_FAULT_WAIT", None)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=root)], env=env, cwd=root, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["async"] == A.AC_ENOMEM, out
    w = workloads.config1()
    a = A.ac_build(w.patterns, alphabet="ACGT")
    d = torch.from_numpy(w.text).cuda()
    d_m = torch.zeros(2 * 8192, dtype=torch.int32, device="cuda")
    d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
    d_c = torch.zeros(a.num_patterns, dtype=torch.int64, device="cuda")
    A.ac_scan_async(a, d, w.text.size, A.AC_U8, None, d_m, 8192, d_num, d_c)
    torch.cuda.synchronize()
    M = int(d_num.item())
    h = hashlib.sha256(d_m.view(-1, 2)[:M].cpu().numpy().tobytes() + d_c.cpu().numpy().tobytes()).hexdigest()
    assert out["noalloc0"] == [M, h] and out["noalloc1"] == [M, h], (out, M)
