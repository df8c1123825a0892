"""Out-of-memory paths on the GPU without a real shortage: AC_FAULT_ALLOC=N
lets N device scratch allocations succeed and fails every later one. Every
call that then misses a buffer reports AC_ENOMEM (nothing is launched on a
missing buffer), the serving loop completes the request with that error,
and the device stays usable. With a few allocations let through, the
failure lands in the middle of a call and is reported the same way. Each
case runs in a child process (the setting is read once per process); no
kernel is made to fault, trap or wait.
"""
import json
import os
import subprocess
import sys

import pytest

from paper_1403_1305_gb300 import ac as A

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
sys.path.insert(0, {root!r})
import torch
import workloads
from paper_1403_1305_gb300 import ac as A
torch.cuda.set_device(0)
w = workloads.config1(n=1 << 16)
a = A.ac_build(w.patterns, alphabet="ACGT")   # its tables come from cudaMalloc, not the scratch pool
d = torch.from_numpy(w.text).cuda()
out = {{}}
def code_of(f):
    try:
        f()
        return 0
    except A.AcError as e:
        return e.code
out["scan_device"] = code_of(lambda: A.ac_scan(a, d))
out["scan_host"] = code_of(lambda: A.ac_scan(a, w.text))
out["batch"] = code_of(lambda: A.ac_scan_batch([a], [(0, d, w.text.size, A.AC_U8)], mem=A.AC_DEVICE))
srv = A.ac_serve_create([a], num_streams=1)
out["serve"] = code_of(lambda: A.ac_serve_wait(srv, A.ac_serve_submit(srv, 0, w.text), 60000))
A.ac_serve_destroy(srv)
out["device_ok"] = torch.ones(1000, device="cuda").sum().item() == 1000.0
print(json.dumps(out))
'''


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(fault):
    env = dict(os.environ)
    env["AC_FAULT_ALLOC"] = str(fault)
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_no_scratch_at_all():
    out = run(0)
    for k in ("scan_device", "scan_host", "batch", "serve"):
        assert out[k] == A.AC_ENOMEM, (k, out)
    assert out["device_ok"]


@pytest.mark.parametrize("fault", [1, 2, 3, 5])
def test_failure_in_the_middle_of_a_call(fault):
    out = run(fault)
    codes = [v for k, v in out.items() if k != "device_ok"]
    assert all(c in (0, A.AC_ENOMEM) for c in codes), out
    assert A.AC_ENOMEM in codes and out["device_ok"]


# Bounded device-side waits run out: AC_FAULT_WAIT=N gives the next N scan
# launches a wait limit of 0, so each gives up at its first mbarrier wait,
# sets the error word, lets the copies it issued land (a bounded wait) and
# exits. The calls report AC_ETIMEDOUT (ac_scan, ac_scan_batch) or write
# UINT64_MAX to *d_num_matches (ac_scan_async); later launches get the normal
# limit and their results equal the oracle's. Nothing waits for something
# that never comes: the copies complete normally, only the wait gives up.
CHILD_WAIT = r'''
import json, sys
sys.path.insert(0, {root!r})
import numpy as np
import torch
import oracle
import workloads
from paper_1403_1305_gb300 import ac as A
torch.cuda.set_device(0)
w = workloads.config2(n=16 << 20, P=2000)       # lean kernel, 16-bit prefix (table copied by one bulk copy)
small = workloads.config1()                      # lean kernel, whole table in shared memory
d = torch.from_numpy(w.text).cuda()
big = A.ac_build(w.patterns, alphabet="ACGT")
few = A.ac_build(small.patterns, alphabet="ACGT")
gen = A.ac_build(w.patterns, alphabet="ACGT")
A.ac_set_scan_config(gen, kernel=A.AC_KERNEL_GENERAL)
n = w.text.size
def code_of(f):
    try:
        f()
        return 0
    except A.AcError as e:
        return e.code
out = {{"kernels": [A.ac_stats(x)["scan_kernel"] for x in (big, few, gen)]}}
out["lean_e16"] = code_of(lambda: A.ac_scan(big, d))
out["lean_smem"] = code_of(lambda: A.ac_scan(few, d))
d_m = torch.empty(1 << 16, dtype=torch.int64, device="cuda")
d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
d_c = torch.empty(gen.num_patterns, dtype=torch.int64, device="cuda")
A.ac_scan_async(gen, d, n, A.AC_U8, None, d_m, 1 << 16, d_num, d_c)
torch.cuda.synchronize()
out["general_async_num"] = int(d_num.item())
out["batch"] = code_of(lambda: A.ac_scan_batch([big], [(0, d, n, A.AC_U8)], mem=A.AC_DEVICE,
                                               flags=A.AC_BATCH_ONE_LAUNCH))
# the limit is back to normal: every path equals the oracle
want = oracle.Machine(w.patterns).scan_mt(w.text, 16)
want_small = oracle.Machine(small.patterns).scan_mt(w.text, 16)
def same(got, exp):
    return bool(np.array_equal(got[0], exp[0]) and np.array_equal(got[1], exp[1]))
out["lean_e16_after"] = same(A.ac_scan(big, d), want)
out["lean_smem_after"] = same(A.ac_scan(few, d), want_small)
out["general_after"] = same(A.ac_scan(gen, d), want)
out["batch_after"] = same(A.ac_scan_batch([big], [(0, d, n, A.AC_U8)], mem=A.AC_DEVICE,
                                          flags=A.AC_BATCH_ONE_LAUNCH)[0], want)
out["device_ok"] = torch.ones(1000, device="cuda").sum().item() == 1000.0
print(json.dumps(out))
'''


def test_bounded_waits_run_out():
    env = dict(os.environ)
    env["AC_FAULT_WAIT"] = "4"
    env.pop("AC_FAULT_ALLOC", None)
    r = subprocess.run([sys.executable, "-c", CHILD_WAIT.format(root=ROOT)], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["kernels"] == [A.AC_KERNEL_LEAN, A.AC_KERNEL_LEAN, A.AC_KERNEL_GENERAL], out
    assert out["lean_e16"] == A.AC_ETIMEDOUT, out
    assert out["lean_smem"] == A.AC_ETIMEDOUT, out
    assert out["general_async_num"] == -1, out   # UINT64_MAX read as int64
    assert out["batch"] == A.AC_ETIMEDOUT, out
    for k in ("lean_e16_after", "lean_smem_after", "general_after", "batch_after", "device_ok"):
        assert out[k] is True, (k, out)
