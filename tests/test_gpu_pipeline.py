"""GPU parity of ac_scan on large host texts, which are copied to the device
in pieces while the pieces already there are scanned (row ranges of one
text geometry per launch), against the oracle, bit-exact.

Cases: pinned and pageable host memory, uint8 and 2-bit packed text, one
machine (lean kernel, warp blocks) and four subsets (CTA tiles), a
protein machine (general kernel), text lengths that leave a partial last
row, and pattern occurrences planted across every piece boundary so that
matches straddle pieces. The same texts scanned from device memory (one
launch) give the same result.
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
MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    yield


def same(got, want):
    gm, gc = got
    wm, wc = want
    assert gm.shape == wm.shape, (gm.shape, wm.shape)
    assert np.array_equal(gm, wm)
    assert np.array_equal(gc, wc)


def plant_across(text, pats, step, rng):
    """Occurrences of random patterns ending just after every multiple of `step` bytes."""
    t = text.copy()
    for b in range(step, t.size, step):
        p = np.frombuffer(pats[int(rng.integers(0, len(pats)))], np.uint8)
        off = int(rng.integers(1, p.size)) if p.size > 1 else 0
        s = b - p.size + off
        if s >= 0 and s + p.size <= t.size:
            t[s:s + p.size] = p
    return t


@pytest.fixture(scope="module")
def dna():
    w = workloads.config2(n=40 * MiB + 12_345)
    rng = np.random.default_rng(1800)
    text = plant_across(w.text, w.patterns, 1 * MiB, rng)
    return w.patterns, text, oracle.Machine(w.patterns).scan_mt(text, THREADS)


@pytest.mark.parametrize("K", [1, 4])
def test_dna_pinned_and_pageable(dna, K):
    pats, text, want = dna
    a = A.ac_build(pats, alphabet="ACGT", num_subsets=K)
    same(A.ac_scan(a, text), want)                                   # pageable
    same(A.ac_scan(a, torch.from_numpy(text).pin_memory(), n=text.size), want)
    same(A.ac_scan(a, torch.from_numpy(text).cuda()), want)          # one launch from device memory


def test_dna_packed_host(dna):
    pats, text, want = dna
    a = A.ac_build(pats, alphabet="ACGT")
    packed = workloads.pack2(text)
    same(A.ac_scan(a, packed, n=text.size, fmt=A.AC_PACKED2), want)
    # a multiple of four symbols short: a partial last byte
    n2 = text.size - 3
    want2 = oracle.Machine(pats).scan_mt(text[:n2], THREADS)
    same(A.ac_scan(a, workloads.pack2(text[:n2]), n=n2, fmt=A.AC_PACKED2), want2)


def test_protein_host_general_kernel():
    w = workloads.config3(n=36 * MiB + 77, P=20_000)
    rng = np.random.default_rng(1801)
    text = plant_across(w.text, w.patterns, 2 * MiB, rng)
    a = A.ac_build(w.patterns, alphabet=w.alphabet)
    assert A.ac_stats(a)["scan_kernel"] == A.AC_KERNEL_GENERAL
    same(A.ac_scan(a, text), oracle.Machine(w.patterns).scan_mt(text, THREADS))


def test_row_length_set_by_the_caller(dna):
    pats, text, want = dna
    a = A.ac_build(pats, alphabet="ACGT")
    for row_len in (96, 1000):
        A.ac_set_scan_config(a, row_len=row_len)
        same(A.ac_scan(a, text), want)
