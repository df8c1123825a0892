"""GPU machine construction (AC_BUILDER_DEVICE) against the host build.

The device builder must produce the host build's machine state for state:
the same breadth-first numbering, folded table with output flags, failure
function, depths and output function (ids ascending per state), for every
subset. Cases: the paper's worked examples, random small pattern sets over
two, four and twenty letters (prefixes, suffixes, duplicates, one-letter
patterns, nested patterns), several subset counts, and the pattern sets of
configs 1-3; then scans of a device-built machine against the oracle.
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


def same_machine(pats, **kw):
    h = A.ac_build(pats, builder=A.AC_BUILDER_HOST, **kw)
    d = A.ac_build(pats, builder=A.AC_BUILDER_DEVICE, **kw)
    sh, sd = A.ac_stats(h), A.ac_stats(d)
    assert sh["states"] == sd["states"] and sh["num_subsets"] == sd["num_subsets"]
    for k in range(sh["num_subsets"]):
        vh, vd = A.ac_subset(h, k), A.ac_subset(d, k)
        for f in ("id_lo", "id_hi", "max_len", "states"):
            assert vh[f] == vd[f], (k, f)
        for f in ("table", "fail", "depth", "out_off", "out_ids", "table16", "table_e16"):
            if vh[f] is None:
                assert vd[f] is None, (k, f)
            else:
                assert np.array_equal(vh[f], vd[f]), (k, f)
    return h, d


def test_worked_examples():
    for pats, text in (([b"AB", b"ABG", b"BEDE", b"EF"], b"ABEDE"),
                       ([b"HE", b"HIS", b"SHE", b"HERS"], b"USHERS")):
        _, d = same_machine(pats)
        m, c = A.ac_scan(d, text)
        wm, wc = oracle.scan(pats, text)
        assert np.array_equal(m, wm) and np.array_equal(c, wc)


@pytest.mark.parametrize("alph", [b"ab", b"ACGT", b"ACDEFGHIKLMNPQRSTVWY"])
def test_random_small_pattern_sets(alph):
    rng = np.random.default_rng(1700 + len(alph))
    for i in range(60):
        text, pats = workloads.tiny_case(rng, alph, max_n=200, max_p=30, max_len=14)
        if i % 7 == 0:
            pats = pats + [pats[0]] * 3 + [alph[:1]]           # duplicates, a one-letter pattern
        if i % 11 == 0:
            pats = pats + [alph[:1] * k for k in range(1, 12)]   # nested
        K = 1 + i % 4 if len(pats) >= 4 else 1
        same_machine(pats, alphabet=alph.decode("latin-1") if i % 2 else None, num_subsets=K)


def test_config_pattern_sets():
    w1 = workloads.config1()
    same_machine(w1.patterns, alphabet="ACGT")
    w2 = workloads.config2(n=4 << 20)
    for K in (1, 16):
        same_machine(w2.patterns, alphabet="ACGT", num_subsets=K)
    w3 = workloads.config3(n=4 << 20)
    same_machine(w3.patterns, alphabet=w3.alphabet)


def test_scans_of_a_device_built_machine():
    w = workloads.config2(n=16 << 20)
    a = A.ac_build(w.patterns, alphabet="ACGT", builder=A.AC_BUILDER_DEVICE)
    d = torch.from_numpy(w.text).cuda()
    m, c = A.ac_scan(a, d)
    wm, wc = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    assert np.array_equal(m, wm) and np.array_equal(c, wc)


def test_device_builder_refusals():
    with pytest.raises(A.AcError):
        A.ac_build([b"ab"], builder=A.AC_BUILDER_DEVICE, machine=A.AC_MACHINE_PFAC)
    with pytest.raises(A.AcError):
        A.ac_build([b"ab"], builder=A.AC_BUILDER_DEVICE, device=-1)
    with pytest.raises(A.AcError):
        A.ac_build([b"ab"], builder=7)

