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
