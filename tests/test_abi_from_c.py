"""The boundary from plain C (CPU only): a C99 program compiled with gcc
against include/ac.h and linked to libacgb300.so builds, saves, loads and
releases automata through the C ABI (no Python between it and the
library)."""
import os
import shutil
import subprocess

import pytest

from paper_1403_1305_gb300 import ac as A

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_uses_the_abi(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no gcc")
    A.lib()  # the library is built
    libdir = os.path.dirname(A.LIB_PATH)
    exe = tmp_path / "abi_from_c"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_from_c.c"),
                        "-L", libdir, "-lacgb300", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe), str(tmp_path / "m.acm")], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.startswith("states 12 ")


@pytest.mark.gpu
def test_c_program_scans_on_the_gpu(tmp_path):
    """A plain C99 program scans the paper's Fig. 1 example on GPU 0 through
    ac_scan, ac_scan_batch and the serving calls (tests/c/scan_from_c.c)."""
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("no gcc")
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A.lib()
    libdir = os.path.dirname(A.LIB_PATH)
    exe = tmp_path / "scan_from_c"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "scan_from_c.c"),
                        "-L", libdir, "-lacgb300", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip().endswith("ok")
