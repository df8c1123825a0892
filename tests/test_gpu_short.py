"""GPU parity of the short-text scan kernel (one thread per row of 16 to 64
bytes, each thread's warm-up and row loaded straight into registers)
against the oracle, bit-exact.

The kernel is forced (AC_KERNEL_SHORT) and also reached through the
automatic choice (texts of at most 8 Mi symbols). Cases: both table placements
(the whole table in shared memory; the escape-coded 16-bit prefix with the
rest read through L2, down to a prefix of a few rows), every row length
and several CTA sizes, text lengths around the 16-byte word and the row
(0, 1, 15, 16, 17, ...), ragged packed tails, bytes outside the alphabet,
a 4-letter alphabet other than ACGT, patterns long enough to need the
nine-word window, rows that begin inside long occurrences, matches at the
first and last positions, host and device texts, a host text long enough
for the pipelined copy (row ranges), the tuner's choice, and refusals where
the kernel does not apply.
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


def fits(pats, row_len):
    """Does a u8 scan's window (warm-up words + row words) fit nine 16-byte words?"""
    warm = max(len(p) for p in pats) - 1
    return (warm + 15) // 16 + max(16, -(-(row_len or 16) // 16) * 16) // 16 <= 9


def all_paths(a, text, want, packed=True):
    """Host bytes, device bytes and (ACGT only) packed host text."""
    text = np.asarray(text, dtype=np.uint8)
    same(A.ac_scan(a, text), want)
    if text.size:
        same(A.ac_scan(a, torch.from_numpy(text.copy()).cuda()), want)
    if packed and not np.any(~np.isin(text, ACGT)):
        same(A.ac_scan(a, workloads.pack2(text), n=text.size, fmt=A.AC_PACKED2), want)


@pytest.mark.parametrize("placement", ["full", "e16"])
def test_random_small_cases(placement):
    rng = np.random.default_rng(1900 + (placement == "e16"))
    for i in range(60):
        text, pats = workloads.tiny_case(rng, b"ACGT", max_n=3000 if i % 4 else 200, max_p=24, max_len=20,
                                         other_frac=0.03 if i % 5 == 0 else 0.0)
        if placement == "e16":
            a = A.ac_build(pats, alphabet="ACGT", placement=A.AC_PLACE_HYBRID16,
                           smem_table_bytes=(16, 64, 256, 4096)[i % 4])
        else:
            a = A.ac_build(pats, alphabet="ACGT")
        row_len = (0, 16, 32, 48, 64)[i % 5]
        A.ac_set_scan_config(a, row_len=row_len, threads=(0, 64, 256, 1024)[i % 4], kernel=A.AC_KERNEL_SHORT)
        if not fits(pats, row_len):      # a pattern longer than the window allows (one longer than the text)
            with pytest.raises(A.AcError) as e:
                A.ac_scan(a, text)
            assert e.value.code == A.AC_EINVAL
            continue
        all_paths(a, text, oracle.scan(pats, text))


def test_lengths_around_words_and_rows():
    rng = np.random.default_rng(1910)
    pats = [b"A", b"AC", b"ACGTACGT", b"T", b"GG", b"TTTTTTTTTTTTTTTTT"]
    for n in [0, 1, 2, 3, 4, 5, 15, 16, 17, 31, 32, 33, 47, 48, 49, 63, 64, 65, 100, 255, 256, 257, 4095, 4097]:
        text = ACGT[rng.integers(0, 4, n)]
        want = oracle.scan(pats, text)
        for row_len in (16, 64):
            a = A.ac_build(pats, alphabet="ACGT")
            A.ac_set_scan_config(a, row_len=row_len, kernel=A.AC_KERNEL_SHORT)
            all_paths(a, text, want)


def test_matches_at_the_first_and_last_positions():
    text = np.frombuffer(b"ACGTTGCA" * 40 + b"GATTACA", np.uint8).copy()
    pats = [b"A", b"AC", b"ACG", b"ACGT", b"GATTACA", b"TACA", b"CA", b"ACGTTGCAACGTTGCAACGTTGCA"]
    a = A.ac_build(pats, alphabet="ACGT")
    A.ac_set_scan_config(a, kernel=A.AC_KERNEL_SHORT)
    all_paths(a, text, oracle.scan(pats, text))


def test_other_four_letter_alphabet():
    """Bytes through the symbol map: a 4-letter alphabet that is not ACGT (the lean kernel does not apply)."""
    rng = np.random.default_rng(1911)
    for i in range(20):
        text, pats = workloads.tiny_case(rng, b"xy01", max_n=2000, max_p=20, max_len=12,
                                         other_frac=0.05 if i % 2 else 0.0)
        a = A.ac_build(pats, alphabet="xy01")
        A.ac_set_scan_config(a, kernel=A.AC_KERNEL_SHORT, row_len=(16, 32)[i % 2])
        if fits(pats, (16, 32)[i % 2]):
            all_paths(a, text, oracle.scan(pats, text), packed=False)
        A.ac_set_scan_config(a)           # the automatic choice on the same text
        same(A.ac_scan(a, text), oracle.scan(pats, text))


@pytest.mark.parametrize("max_len", [40, 64, 100, 120])
def test_long_patterns_need_the_wide_window(max_len):
    rng = np.random.default_rng(1920 + max_len)
    text = ACGT[rng.integers(0, 4, 50_000)]
    pats = [text[o:o + L].tobytes() for o, L in
            ((int(rng.integers(0, text.size - max_len)), int(rng.integers(max_len // 2, max_len + 1)))
             for _ in range(200))]
    pats.append(text[100:100 + max_len].tobytes())
    want = oracle.scan(pats, text)
    for row_len in (16, 64):
        a = A.ac_build(pats, alphabet="ACGT")
        A.ac_set_scan_config(a, kernel=A.AC_KERNEL_SHORT, row_len=row_len)
        if not fits(pats, row_len):
            with pytest.raises(A.AcError) as e:
                A.ac_scan(a, text)
            assert e.value.code == A.AC_EINVAL
            continue
        all_paths(a, text, want)


@pytest.mark.parametrize("L", [17, 18, 24, 32, 33, 34, 48, 49])
def test_rows_begin_inside_long_occurrences(L):
    """Rows of 16 bytes that begin inside long occurrences (runs of one
    letter, planted copies of the longest patterns), so that a row's warm-up
    must carry a deep state into it, for longest-pattern lengths on both
    sides of multiples of the 16-byte word."""
    rng = np.random.default_rng(1940 + L)
    text = ACGT[rng.integers(0, 4, 60_000)]
    text[1000:1400] = ord("A")                      # a run: deep states at many row starts
    text[5003:5003 + 3 * L] = ord("C")
    pats = [b"A" * L, b"C" * (L - 1), b"ACGT"]
    pats += [text[o:o + L].tobytes() for o in rng.integers(0, text.size - L, 20)]
    pats += [text[o:o + n].tobytes() for o, n in zip(rng.integers(0, text.size - L, 30), rng.integers(4, L, 30))]
    text = workloads.embed(rng, text, pats[3:23], 400)
    want = oracle.scan(pats, text)
    a = A.ac_build(pats, alphabet="ACGT")
    for threads in (64, 512, 1024):
        A.ac_set_scan_config(a, kernel=A.AC_KERNEL_SHORT, row_len=16, threads=threads)
        all_paths(a, text, want)
    a16 = A.ac_build(pats, alphabet="ACGT", placement=A.AC_PLACE_HYBRID16, smem_table_bytes=256)
    A.ac_set_scan_config(a16, kernel=A.AC_KERNEL_SHORT, row_len=16)
    all_paths(a16, text, want)


@pytest.mark.parametrize("config", ["config1", "config2"])
def test_configs_automatic_choice(config):
    """Config 1 (whole table in shared memory) and a 4 MiB config-2 text
    (344k states: the 16-bit prefix and L2) through the automatic choice,
    which takes the short-text kernel at these sizes."""
    w = workloads.config1() if config == "config1" else workloads.config2(n=4 << 20)
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    a = A.ac_build(w.patterns, alphabet="ACGT")
    all_paths(a, w.text, want)
    A.ac_set_scan_config(a, kernel=A.AC_KERNEL_SHORT, threads=1024)
    all_paths(a, w.text, want)
    A.ac_set_scan_config(a, kernel=A.AC_KERNEL_LEAN)
    same(A.ac_scan(a, torch.from_numpy(w.text).cuda()), want)


def test_long_host_text_in_pieces():
    """A forced short-text scan of a 34 MiB host text is copied and scanned in
    pieces (row ranges of 16-byte rows); matches straddle the pieces."""
    w = workloads.config2(n=34 * (1 << 20) + 5)
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    a = A.ac_build(w.patterns, alphabet="ACGT")
    A.ac_set_scan_config(a, kernel=A.AC_KERNEL_SHORT)
    same(A.ac_scan(a, w.text), want)


def test_tuner_on_a_short_text():
    w = workloads.config1()
    a = A.ac_build(w.patterns, alphabet="ACGT")
    d = torch.from_numpy(w.text).cuda()
    cfg = A.ac_tune(a, d)
    assert cfg["kernel"] in (A.AC_KERNEL_GENERAL, A.AC_KERNEL_LEAN, A.AC_KERNEL_SHORT)
    same(A.ac_scan(a, d), oracle.scan(w.patterns, w.text))


def test_refusals():
    rng = np.random.default_rng(1930)
    text = ACGT[rng.integers(0, 4, 1000)]
    pats = [b"ACG", b"GT", b"TTA", b"CAT"]
    a = A.ac_build(pats, alphabet="ACGT", num_subsets=2)      # pattern subsets
    A.ac_set_scan_config(a, kernel=A.AC_KERNEL_SHORT)
    with pytest.raises(A.AcError) as e:
        A.ac_scan(a, text)
    assert e.value.code == A.AC_EINVAL
    A.ac_set_scan_config(a)                                   # the automatic choice steps aside
    same(A.ac_scan(a, text), oracle.scan(pats, text))
    b = A.ac_build(pats, alphabet="ACGT")
    for kw in (dict(threads=32), dict(row_len=80), dict(chains=2)):
        A.ac_set_scan_config(b, kernel=A.AC_KERNEL_SHORT, **kw)
        with pytest.raises(A.AcError) as e:
            A.ac_scan(b, text)
        assert e.value.code == A.AC_EINVAL
    p = A.ac_build([b"ACD", b"WY"], alphabet=workloads.PROTEIN)   # 20 letters
    A.ac_set_scan_config(p, kernel=A.AC_KERNEL_SHORT)
    with pytest.raises(A.AcError) as e:
        A.ac_scan(p, b"ACDWY")
    assert e.value.code == A.AC_EINVAL


def async_scan(a, d_text, n, cap, fmt=A.AC_U8):
    d_m = torch.full((2 * max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    d_num = torch.full((1,), 777, dtype=torch.int64, device="cuda")
    d_c = torch.full((a.num_patterns,), 5, dtype=torch.int64, device="cuda")
    A.ac_scan_async(a, d_text, n, fmt, None, d_m, cap, d_num, d_c)
    torch.cuda.synchronize()
    M = int(d_num.item())
    return M, d_m.view(-1, 2)[:min(M, cap)].cpu().numpy().view(np.uint32), d_c.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("placement", ["full", "e16"])
def test_async_small_capacities(placement):
    """ac_scan_async on short texts with capacities of 1..2,048 records
    (the rank sort), results of 0..~1,900 matches, packed and byte text;
    with M > cap the count and the counts are still exact."""
    rng = np.random.default_rng(1700 + (placement == "e16"))
    for i, (n, P, cap) in enumerate(((20_000, 40, 2048), (50_000, 300, 1024), (3_000, 10, 64), (120_000, 200, 2048),
                                     (1, 5, 1), (700_000, 100, 2048), (9_000, 60, 7))):
        text = workloads.dna_text(rng, n)
        pats = workloads.draw_patterns(rng, text, P, 4 if i % 2 else 6, 16, 0.9, ACGT)
        kw = dict(placement=A.AC_PLACE_HYBRID16, smem_table_bytes=512) if placement == "e16" else {}
        a = A.ac_build(pats, alphabet="ACGT", **kw)
        assert A.ac_stats(a)["scan_kernel"] in (A.AC_KERNEL_SHORT, A.AC_KERNEL_LEAN)
        wm, wc = oracle.scan(pats, text)
        for fmt, t in ((A.AC_U8, text), (A.AC_PACKED2, workloads.pack2(text))):
            M, m, c = async_scan(a, torch.from_numpy(np.ascontiguousarray(t)).cuda(), n, cap, fmt)
            assert M == wm.shape[0]
            assert np.array_equal(c, wc)
            if M <= cap:
                assert np.array_equal(m, wm)
