"""GPU parity of the two-symbol-table scan (one lookup per two DNA symbols)
against the oracle, bit-exact, next to the one-symbol scan of the same
automaton.

Cases: odd and even text lengths (a ragged last symbol), bytes outside ACGT,
packed text, isolated matches ending at even and at odd positions (the
direct emit of a single flagged step and the pair-wise careful walk), a
match at every position, chain rows short enough that matches straddle
them, shared-memory budgets down to nothing (every lookup through L2), and
several subset counts (one machine: flag tracking on; many: off).
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
ACGT = np.frombuffer(b"ACGT", np.uint8)


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


def both_strides(a, text, want, packed=True, **cfg):
    for stride in (1, 2):
        A.ac_set_scan_config(a, stride=stride, **cfg)
        same(A.ac_scan(a, text), want)
        if packed and not np.any(~np.isin(np.asarray(text), ACGT)):
            same(A.ac_scan(a, workloads.pack2(np.asarray(text)), n=len(text), fmt=A.AC_PACKED2), want)


CONFIGS = [
    dict(row_len=32, threads=32, chains=1),
    dict(row_len=64, threads=64, chains=2, stage_bytes=16),
    dict(row_len=96, threads=128, chains=4, stage_bytes=16),
    dict(row_len=128, threads=256, chains=2, stage_bytes=32, ctas=5),
    dict(),
]


@pytest.mark.parametrize("cfg", range(len(CONFIGS)))
def test_random_small_cases(cfg):
    rng = np.random.default_rng(600 + cfg)
    for i in range(80):
        text, pats = workloads.tiny_case(rng, b"ACGT", max_n=900, max_p=16, max_len=20,
                                         other_frac=0.03 if i % 4 == 0 else 0.0)
        K = 1 + i % 3 if len(pats) >= 3 else 1
        a = A.ac_build(pats, alphabet="ACGT", num_subsets=K, stride=2,
                       smem_table_bytes=(0, 64, 2048)[i % 3])
        both_strides(a, np.asarray(text), oracle.scan(pats, text), **CONFIGS[cfg])


@pytest.mark.parametrize("K", [1, 3])
def test_isolated_matches_at_even_and_odd_ends(K):
    """Few matches, far apart: a stage holds at most one flagged step, at the
    first or the second symbol of a pair."""
    rng = np.random.default_rng(610 + K)
    for n in (20_001, 20_000, 65_537):
        text = workloads.dna_text(rng, n)
        pats = [bytes(workloads.dna_text(rng, int(rng.integers(9, 21)))) for _ in range(12)]
        for j, p in enumerate(pats):
            for _ in range(3):
                end = int(rng.integers(len(p), n))
                end += (end + j) % 2  # alternate end parity over the patterns
                if end < n:
                    text[end - len(p) + 1:end + 1] = np.frombuffer(p, np.uint8)
        want = oracle.scan(pats, text)
        assert want[0].shape[0] >= 20
        assert len(set((want[0][:, 0] % 2).tolist())) == 2
        a = A.ac_build(pats, alphabet="ACGT", num_subsets=K, stride=2)
        both_strides(a, text, want, row_len=512, threads=128, chains=2)
        both_strides(a, text, want)


@pytest.mark.parametrize("K", [1, 4])
def test_match_at_every_position(K):
    import itertools
    pats = [bytes(p) for p in itertools.product(b"ACGT", repeat=3)] + [b"A", b"CG", b"ACGTACGT"]
    rng = np.random.default_rng(620 + K)
    for n in (7, 64, 1001, 30_000):
        text = workloads.dna_text(rng, n)
        a = A.ac_build(pats, alphabet="ACGT", num_subsets=K, stride=2)
        both_strides(a, text, oracle.scan(pats, text), row_len=64, threads=64, chains=2)


def test_global_placement_and_bytes_outside_the_alphabet():
    rng = np.random.default_rng(630)
    text = workloads.dna_text(rng, 100_001)
    pats = workloads.draw_patterns(rng, text, 400, 4, 24, 0.7, ACGT)
    for other in (b"N", b"a", b"\x00"):
        t = text.copy()
        t[rng.random(t.size) < 0.002] = other[0]
        want = oracle.scan(pats, t)
        for placement in (A.AC_PLACE_AUTO, A.AC_PLACE_GLOBAL, A.AC_PLACE_HYBRID):
            a = A.ac_build(pats, alphabet="ACGT", placement=placement, smem_table_bytes=4096, stride=2)
            both_strides(a, t, want, packed=False, row_len=256, threads=128, chains=2)


def test_ragged_lengths_u8_and_packed():
    rng = np.random.default_rng(640)
    for n in list(range(1, 40)) + [63, 64, 65, 127, 129, 255, 257, 4093, 4099]:
        text = workloads.dna_text(rng, n)
        src = workloads.dna_text(rng, 64)
        pats = workloads.draw_patterns(rng, [src, text], 16, 1, 7, 0.6, ACGT)
        a = A.ac_build(pats, alphabet="ACGT", stride=2)
        both_strides(a, text, oracle.scan(pats, text), row_len=64, threads=32, chains=2, stage_bytes=16)


def test_automatic_stride():
    """Two symbols per lookup by default only where they pay: config 2 at 16
    subsets (built and chosen), not at one machine (not even built)."""
    w = workloads.config2(n=4 << 20)
    a16 = A.ac_build(w.patterns, alphabet="ACGT", num_subsets=16)
    st = A.ac_stats(a16)
    assert st["table2_bytes"] > 0 and st["scan_stride"] == 2
    a1 = A.ac_build(w.patterns, alphabet="ACGT")
    st = A.ac_stats(a1)
    assert st["table2_bytes"] == 0 and st["scan_stride"] == 1
    assert st["scan_placement"] == A.AC_PLACE_HYBRID16
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    d = torch.from_numpy(w.text).cuda()
    same(A.ac_scan(a16, d), want)
    same(A.ac_scan(a1, d), want)


def test_stride_selection_and_errors():
    rng = np.random.default_rng(650)
    text = workloads.dna_text(rng, 5000)
    pats = workloads.draw_patterns(rng, text, 30, 4, 12, 0.8, ACGT)
    want = oracle.scan(pats, text)
    # a 4-letter alphabet that is not ACGT: byte text scans with stride 1
    # (asked for 2: AC_EINVAL), packed text with 2
    low = [p.lower() for p in pats]
    tl = np.frombuffer(bytes(text).lower(), np.uint8)
    a = A.ac_build(low, alphabet="acgt", stride=2)
    same(A.ac_scan(a, tl), want)
    A.ac_set_scan_config(a, stride=2)
    with pytest.raises(A.AcError) as e:
        A.ac_scan(a, tl)
    assert e.value.code == A.AC_EINVAL
    same(A.ac_scan(a, workloads.pack2(text), n=text.size, fmt=A.AC_PACKED2), want)
    # built without the two-symbol table
    a = A.ac_build(pats, alphabet="ACGT", stride=1)
    same(A.ac_scan(a, text), want)
    with pytest.raises(A.AcError):
        A.ac_set_scan_config(a, stride=2)
    # placement SMEM: the one-symbol table fits, the two-symbol one does not,
    # so the automatic stride falls back to 1
    w = workloads.config2(n=1 << 20, P=200)
    a = A.ac_build(w.patterns, alphabet="ACGT", placement=A.AC_PLACE_SMEM, stride=2)
    st = A.ac_stats(a)
    assert st["table_bytes"] < (128 << 10) and st["table2_bytes"] > (232 << 10)
    same(A.ac_scan(a, w.text), oracle.scan(w.patterns, w.text))
    A.ac_set_scan_config(a, stride=2)
    with pytest.raises(A.AcError) as e:
        A.ac_scan(a, w.text)
    assert e.value.code == A.AC_ERANGE


@pytest.fixture(scope="module")
def cfg2_small():
    return workloads.config2(n=16 << 20)


@pytest.mark.parametrize("K", [1, 4, 16, 64])
def test_config2_16MiB_both_strides(cfg2_small, K):
    w = cfg2_small
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    a = A.ac_build(w.patterns, alphabet="ACGT", num_subsets=K, stride=2)
    d = torch.from_numpy(w.text).cuda()
    dp = torch.from_numpy(workloads.pack2(w.text)).cuda()
    for stride in (1, 2):
        A.ac_set_scan_config(a, stride=stride)
        same(A.ac_scan(a, d), want)
        same(A.ac_scan(a, dp, n=w.text.size, fmt=A.AC_PACKED2), want)


def test_config2_full_size_embedded_matches():
    """256 MiB DNA, 10,000 patterns, 100,000 embedded occurrences: dense
    enough that many stages take the careful walk."""
    w = workloads.config2()
    rng = np.random.default_rng(660)
    text = workloads.embed(rng, w.text.copy(), w.patterns, 100_000)
    want = oracle.Machine(w.patterns).scan_mt(text, THREADS)
    a = A.ac_build(w.patterns, alphabet="ACGT", stride=2)
    d = torch.from_numpy(text).cuda()
    for stride in (2, 1):
        A.ac_set_scan_config(a, stride=stride)
        same(A.ac_scan(a, d), want)
