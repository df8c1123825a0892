"""An automaton saved with ac_save and loaded onto the GPU with ac_load:
its tables equal the built one's and its scans give the oracle's result.
"""
import os

import numpy as np
import pytest

import oracle
import workloads
from paper_1403_1305_gb300 import ac as A

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    yield


def test_saved_and_loaded_machine_scans_the_same(tmp_path):
    """ac_save, then ac_load onto the GPU: the loaded automaton's tables equal
    the built one's and its scans give the oracle's result (one machine and
    four subsets, byte and packed text)."""
    w = workloads.config2(n=4 << 20)
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    d = torch.from_numpy(w.text).cuda()
    for K in (1, 4):
        a = A.ac_build(w.patterns, alphabet="ACGT", num_subsets=K)
        path = tmp_path / f"config2_k{K}.acm"
        A.ac_save(a, path)
        b = A.ac_load(path, device=0)
        for k in range(K):
            va, vb = A.ac_subset(a, k), A.ac_subset(b, k)
            for f in ("table", "out_off", "out_ids", "table_e16"):
                assert (va[f] is None and vb[f] is None) or np.array_equal(va[f], vb[f]), (K, f)
        m, c = A.ac_scan(b, d)
        assert np.array_equal(m, want[0]) and np.array_equal(c, want[1])
        m, c = A.ac_scan(b, workloads.pack2(w.text), n=w.text.size, fmt=A.AC_PACKED2)
        assert np.array_equal(m, want[0]) and np.array_equal(c, want[1])
