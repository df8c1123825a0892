"""GPU parity of the lean scan kernel (one-symbol tables of a 4-letter
machine over ACGT bytes or 2-bit packed text) against the oracle, bit-exact.

The kernel is forced (AC_KERNEL_LEAN) in each of its CTA shapes and both of
its table placements: every row in shared memory as 32-bit row offsets, and
the escape-coded 16-bit prefix with the rest read through L2 (forced with
AC_PLACE_HYBRID16 and small shared-memory caps, down to a prefix of a few
rows so most lookups go to L2). Cases: short rows so matches straddle chain
rows and warp blocks, one machine (warps take their own row blocks) and
several subsets (CTA tiles), odd text lengths and ragged packed tails,
bytes outside ACGT, unaligned device texts, nested patterns whose output
holds many suffixes, a match at every position, and config 1 / config 2 at
the bench's sizes next to the general kernel.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import workloads
from paper_1403_1305_gb300 import ac as A

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4
ACGT = np.frombuffer(b"ACGT", np.uint8)
SHAPES = [(1024, 4), (1024, 3), (1024, 2), (768, 4), (512, 4)]


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


def both_formats(a, text, want):
    same(A.ac_scan(a, text), want)
    text = np.asarray(text)
    if not np.any(~np.isin(text, ACGT)):
        same(A.ac_scan(a, workloads.pack2(text), n=text.size, fmt=A.AC_PACKED2), want)


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("placement", ["smem32", "e16"])
def test_random_small_cases(shape, placement):
    threads, chains = SHAPES[shape]
    rng = np.random.default_rng(1100 + 10 * shape + (placement == "e16"))
    for i in range(40):
        text, pats = workloads.tiny_case(rng, b"ACGT", max_n=3000 if i % 4 else 300, max_p=24, max_len=20,
                                         other_frac=0.03 if i % 5 == 0 else 0.0)
        K = 1 + (i % 3) if len(pats) >= 3 else 1
        if placement == "e16":
            a = A.ac_build(pats, alphabet="ACGT", num_subsets=K, placement=A.AC_PLACE_HYBRID16,
                           smem_table_bytes=(64, 256, 4096)[i % 3])
        else:
            a = A.ac_build(pats, alphabet="ACGT", num_subsets=K)
        A.ac_set_scan_config(a, row_len=(32, 64, 96, 160, 0)[i % 5], threads=threads, chains=chains,
                             kernel=A.AC_KERNEL_LEAN)
        st = A.ac_stats(a)
        assert st["scan_kernel"] == A.AC_KERNEL_LEAN
        if placement == "e16":
            assert st["scan_placement"] == A.AC_PLACE_HYBRID16
        else:   # whole table in shared memory unless it is too large (a pattern longer than the text)
            if st["scan_placement"] == A.AC_PLACE_SMEM:
                assert st["smem_states"] == st["states"]
            else:
                assert st["scan_placement"] == A.AC_PLACE_HYBRID16 and st["states"] * 16 > 100_000
        both_formats(a, text, oracle.scan(pats, text))


def test_default_kernel_is_lean_for_dna():
    rng = np.random.default_rng(1200)
    text = workloads.dna_text(rng, 20_000)
    pats = workloads.draw_patterns(rng, text, 100, 8, 32, 0.5, ACGT)
    a = A.ac_build(pats, alphabet="ACGT")
    st = A.ac_stats(a)
    assert st["scan_placement"] == A.AC_PLACE_SMEM and st["smem_states"] == st["states"]
    both_formats(a, text, oracle.scan(pats, text))
    # the general kernel on the same automaton
    A.ac_set_scan_config(a, kernel=A.AC_KERNEL_GENERAL)
    both_formats(a, text, oracle.scan(pats, text))


def test_lean_refuses_what_it_cannot_scan():
    pats = [b"ACDE", b"KLM"]
    a = A.ac_build(pats)
    A.ac_set_scan_config(a, kernel=A.AC_KERNEL_LEAN)
    with pytest.raises(A.AcError):
        A.ac_scan(a, b"ACDEKLM")
    a = A.ac_build([b"ACG", b"GT"], alphabet="ACGT")
    A.ac_set_scan_config(a, kernel=A.AC_KERNEL_LEAN, threads=256, chains=2)
    with pytest.raises(A.AcError):
        A.ac_scan(a, b"ACGTACGT")
    # automatic choice falls back to the general kernel for such shapes
    A.ac_set_scan_config(a, threads=256, chains=2)
    same(A.ac_scan(a, b"ACGTACGT"), oracle.scan([b"ACG", b"GT"], b"ACGTACGT"))


@pytest.mark.parametrize("cap", [64, 2048, 0])
def test_escape_prefix_sizes(cap):
    """E16 with prefixes from a few rows to all of shared memory; nested
    patterns (A, AA, ..., A^30) make outputs at shallow states (escapes)."""
    rng = np.random.default_rng(1300 + cap)
    nested = [b"A" * k for k in range(1, 31)]
    for i in range(12):
        text = workloads.dna_text(rng, int(rng.integers(1, 20_000)))
        if i % 3 == 0:
            text[rng.random(text.size) < 0.3] = ord("A")
        pats = workloads.draw_patterns(rng, text, 300, 4, 24, 0.6, ACGT) + (nested if i % 2 else [])
        a = A.ac_build(pats, alphabet="ACGT", placement=A.AC_PLACE_HYBRID16, smem_table_bytes=cap)
        A.ac_set_scan_config(a, row_len=(64, 128, 0)[i % 3], kernel=A.AC_KERNEL_LEAN)
        both_formats(a, text, oracle.scan(pats, text))


def test_every_position_matches_and_ragged_packed():
    pats = [bytes(p) for p in itertools.product(b"ACGT", repeat=3)]
    a = A.ac_build(pats, alphabet="ACGT")
    rng = np.random.default_rng(1400)
    for n in list(range(0, 70)) + [127, 128, 129, 4093, 4096, 4099, 100_001]:
        text = workloads.dna_text(rng, n)
        A.ac_set_scan_config(a, row_len=64 if n % 2 else 0, kernel=A.AC_KERNEL_LEAN)
        both_formats(a, text, oracle.scan(pats, text))


def test_bytes_outside_acgt_and_unaligned_device_text():
    rng = np.random.default_rng(1500)
    text = workloads.dna_text(rng, 60_000)
    pats = workloads.draw_patterns(rng, text, 400, 4, 20, 0.8, ACGT)
    for place in (A.AC_PLACE_AUTO, A.AC_PLACE_HYBRID16):
        a = A.ac_build(pats, alphabet="ACGT", placement=place, smem_table_bytes=1024 if place else 0)
        A.ac_set_scan_config(a, row_len=96, kernel=A.AC_KERNEL_LEAN)
        for other in (b"N", b"a", b"\x00", b"\xff", b"\n"):
            t = text.copy()
            t[rng.random(t.size) < 0.01] = other[0]
            same(A.ac_scan(a, t), oracle.scan(pats, t))
        want = oracle.scan(pats, text)
        src = torch.from_numpy(text).cuda()
        for off in (0, 1, 3, 15, 16):
            buf = torch.zeros(text.size + 64, dtype=torch.uint8, device="cuda")
            view = buf[off:off + text.size]
            view.copy_(src)
            same(A.ac_scan(a, view), want)


def test_config1_full_and_row_lengths():
    w = workloads.config1()
    want = oracle.scan(w.patterns, w.text)
    a = A.ac_build(w.patterns, alphabet="ACGT")
    d = torch.from_numpy(w.text).cuda()
    for shape in SHAPES:
        for row_len in (64, 256, 0):
            A.ac_set_scan_config(a, row_len=row_len, threads=shape[0], chains=shape[1], kernel=A.AC_KERNEL_LEAN)
            same(A.ac_scan(a, d), want)


@pytest.fixture(scope="module")
def cfg2_small():
    return workloads.config2(n=16 << 20)


@pytest.mark.parametrize("K", [1, 4, 16, 64])
def test_config2_subsets_16MiB(cfg2_small, K):
    w = cfg2_small
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    d = torch.from_numpy(w.text).cuda()
    dp = torch.from_numpy(workloads.pack2(w.text)).cuda()
    for place in (A.AC_PLACE_AUTO, A.AC_PLACE_HYBRID16):
        a = A.ac_build(w.patterns, alphabet="ACGT", num_subsets=K, placement=place, stride=1)
        for shape in ((1024, 4), (768, 4)):
            A.ac_set_scan_config(a, threads=shape[0], chains=shape[1], kernel=A.AC_KERNEL_LEAN)
            same(A.ac_scan(a, d), want)
            same(A.ac_scan(a, dp, n=w.text.size, fmt=A.AC_PACKED2), want)
