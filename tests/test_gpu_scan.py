"""GPU parity: the CUDA scan (through the C ABI) against the oracle, bit-exact.

Every comparison is element by element on the sorted (end position, pattern
id) list and on the per-pattern counts; the oracle runs on the same seeded
inputs. Small cases force short chain rows so matches straddle chain
boundaries, tiny shared-memory budgets so lookups go through L2, several
subset counts, both text formats, device inputs at unaligned addresses,
bytes outside the alphabet, empty and ragged texts. The full-size cases run
at the sizes and launch configuration of bench.py.
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


def same(got, want):
    gm, gc = got
    wm, wc = want
    assert gm.shape == wm.shape, (gm.shape, wm.shape)
    assert np.array_equal(gm, wm)
    assert np.array_equal(gc, wc)


def test_worked_examples():
    for pats, text in (([b"AB", b"ABG", b"BEDE", b"EF"], b"ABEDE"),
                       ([b"HE", b"HIS", b"SHE", b"HERS"], b"USHERS")):
        a = A.ac_build(pats)
        same(A.ac_scan(a, text), oracle.scan(pats, text))
        d = torch.frombuffer(bytearray(text), dtype=torch.uint8).cuda()
        same(A.ac_scan(a, d), oracle.scan(pats, text))


CONFIGS = [
    dict(row_len=16, threads=32, chains=1),
    dict(row_len=32, threads=64, chains=2),
    dict(row_len=48, threads=128, chains=4),
    dict(row_len=64, threads=256, chains=4, ctas=3),
    dict(row_len=0, threads=0, chains=0),
    dict(row_len=32, threads=64, chains=2, stage_bytes=16),
    dict(row_len=80, threads=128, chains=4, stage_bytes=16),
]


@pytest.mark.parametrize("cfg", range(len(CONFIGS)))
def test_random_small_cases(cfg):
    rng = np.random.default_rng(200 + cfg)
    for i in range(120):
        alph = (b"ACGT", b"ab", b"ACDEFGHIKLMNPQRSTVWY")[i % 3]
        text, pats = workloads.tiny_case(rng, alph, max_n=400, max_p=12, max_len=24,
                                         other_frac=0.05 if i % 5 == 0 else 0.0)
        K = 1 + (i % 3) if len(pats) >= 3 else 1
        a = A.ac_build(pats, num_subsets=K)
        A.ac_set_scan_config(a, **CONFIGS[cfg])
        same(A.ac_scan(a, text), oracle.scan(pats, text))


@pytest.mark.parametrize("smem", [16, 256, 4096])
def test_hybrid_and_global_placement(smem):
    """Tiny shared-memory budgets push most lookups through L2."""
    rng = np.random.default_rng(300 + smem)
    for i in range(60):
        text, pats = workloads.tiny_case(rng, b"ACGT", max_n=700, max_p=30, max_len=12, other_frac=0.02)
        a = A.ac_build(pats, alphabet="ACGT", placement=A.AC_PLACE_HYBRID, smem_table_bytes=smem)
        A.ac_set_scan_config(a, row_len=32, threads=64, chains=2, stage_bytes=16 if i % 2 else 32)
        same(A.ac_scan(a, text), oracle.scan(pats, text))
    a = A.ac_build(pats, alphabet="ACGT", placement=A.AC_PLACE_GLOBAL)
    same(A.ac_scan(a, text), oracle.scan(pats, text))


def test_packed_text_ragged_lengths():
    rng = np.random.default_rng(9)
    for n in list(range(0, 70)) + [127, 128, 129, 255, 256, 257, 1000, 4093, 4096, 4099]:
        text = workloads.dna_text(rng, n)
        src = text if n >= 64 else workloads.dna_text(rng, 64)
        pats = workloads.draw_patterns(rng, [src, text] if n else src, 20, 1, 9, 0.5,
                                       np.frombuffer(b"ACGT", np.uint8))
        a = A.ac_build(pats, alphabet="ACGT")
        A.ac_set_scan_config(a, row_len=128, threads=64, chains=2, stage_bytes=16 if n % 2 else 32)
        want = oracle.scan(pats, text)
        packed = workloads.pack2(text)
        same(A.ac_scan(a, packed, n=n, fmt=A.AC_PACKED2), want)
        same(A.ac_scan(a, text), want)


def test_bytes_outside_the_alphabet():
    rng = np.random.default_rng(10)
    text = workloads.dna_text(rng, 50_000)
    pats = workloads.draw_patterns(rng, text, 200, 4, 20, 0.8, np.frombuffer(b"ACGT", np.uint8))
    for other in (b"N", b"a", b"\x00", b"\xff", b"\n"):
        t = text.copy()
        t[rng.random(t.size) < 0.01] = other[0]
        a = A.ac_build(pats, alphabet="ACGT")
        A.ac_set_scan_config(a, row_len=256, threads=128, chains=2)
        same(A.ac_scan(a, t), oracle.scan(pats, t))


def test_device_input_unaligned_and_async():
    rng = np.random.default_rng(11)
    text = workloads.dna_text(rng, 100_003)
    pats = workloads.draw_patterns(rng, text, 300, 6, 30, 0.5, np.frombuffer(b"ACGT", np.uint8))
    a = A.ac_build(pats, alphabet="ACGT")
    want = oracle.scan(pats, text)
    src = torch.from_numpy(text).cuda()
    for off in (0, 1, 3, 8, 15, 16, 31):
        buf = torch.zeros(text.size + 64, dtype=torch.uint8, device="cuda")
        view = buf[off:off + text.size]
        view.copy_(src)
        same(A.ac_scan(a, view), want)
    # asynchronous device-in device-out path, and its two stages
    dt = torch.from_numpy(text).cuda()
    M = want[0].shape[0]
    cap = M + 17
    d_m = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
    d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
    d_c = torch.zeros(a.num_patterns, dtype=torch.int64, device="cuda")
    A.ac_scan_async(a, dt, text.size, A.AC_U8, None, d_m, cap, d_num, d_c)
    torch.cuda.synchronize()
    assert int(d_num.item()) == M
    got = d_m.view(-1, 2)[:M].cpu().numpy().view(np.uint32)
    same((got, d_c.cpu().numpy().view(np.uint64)), want)
    # too small a capacity: the true count comes back
    A.ac_scan_async(a, dt, text.size, A.AC_U8, None, d_m, max(1, M // 2), d_num, None)
    torch.cuda.synchronize()
    assert int(d_num.item()) == M


def test_empty_and_degenerate():
    a = A.ac_build([b"ACGT", b"A"], alphabet="ACGT")
    m, c = A.ac_scan(a, b"")
    assert m.shape == (0, 2) and c.tolist() == [0, 0]
    same(A.ac_scan(a, b"A"), oracle.scan([b"ACGT", b"A"], b"A"))
    same(A.ac_scan(a, b"ACG"), oracle.scan([b"ACGT", b"A"], b"ACG"))
    long_pat = [b"ACGT" * 40]
    a = A.ac_build(long_pat)
    A.ac_set_scan_config(a, row_len=16, threads=32, chains=1)
    txt = b"ACGT" * 100
    same(A.ac_scan(a, txt), oracle.scan(long_pat, txt))
    # duplicates: every id reported
    pats = [b"AC", b"AC", b"C", b"ACAC"]
    a = A.ac_build(pats)
    same(A.ac_scan(a, b"ACACAC" * 50), oracle.scan(pats, b"ACACAC" * 50))
    # a pattern whose output includes many suffixes (a, aa, aaa, ...)
    pats = [b"a" * k for k in range(1, 40)]
    a = A.ac_build(pats)
    A.ac_set_scan_config(a, row_len=32, threads=64, chains=2)
    same(A.ac_scan(a, b"a" * 5000), oracle.scan(pats, b"a" * 5000))


def test_row_length_invariance_config1():
    w = workloads.config1()
    want = oracle.scan(w.patterns, w.text)
    a = A.ac_build(w.patterns, alphabet="ACGT")
    for row_len in (32, 96, 256, 1024, 0):
        A.ac_set_scan_config(a, row_len=row_len)
        same(A.ac_scan(a, w.text), want)


def test_config1_full():
    w = workloads.config1()
    a = A.ac_build(w.patterns, alphabet="ACGT")
    same(A.ac_scan(a, torch.from_numpy(w.text).cuda()), oracle.scan(w.patterns, w.text))


@pytest.fixture(scope="module")
def cfg2_small():
    return workloads.config2(n=16 << 20)


@pytest.mark.parametrize("K", [1, 4, 16, 64])
def test_config2_subsets_16MiB(cfg2_small, K):
    w = cfg2_small
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    a = A.ac_build(w.patterns, alphabet="ACGT", num_subsets=K)
    d = torch.from_numpy(w.text).cuda()
    same(A.ac_scan(a, d), want)
    same(A.ac_scan(a, torch.from_numpy(workloads.pack2(w.text)).cuda(), n=w.text.size, fmt=A.AC_PACKED2), want)


def test_config2_full_size():
    """256 MiB DNA, 10,000 patterns: bench.py's workload and launch configuration."""
    w = workloads.config2()
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    a = A.ac_build(w.patterns, alphabet="ACGT")
    d = torch.from_numpy(w.text).cuda()
    same(A.ac_scan(a, d), want)
    same(A.ac_scan(a, torch.from_numpy(workloads.pack2(w.text)).cuda(), n=w.text.size, fmt=A.AC_PACKED2), want)


def test_config3_full_size():
    """64 MiB protein text, 100,000 patterns: the table does not fit in shared memory."""
    w = workloads.config3()
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    a = A.ac_build(w.patterns, alphabet=w.alphabet)
    st = A.ac_stats(a)
    assert st["smem_states"] < st["states"]
    same(A.ac_scan(a, torch.from_numpy(w.text).cuda()), want)


def test_failure_less_machine_scan():
    """The paper's own method on the GPU (AC_MACHINE_PFAC): same results."""
    rng = np.random.default_rng(71)
    for i in range(150):
        alph = (b"ACGT", b"ab", b"ACDEFGHIKLMNPQRSTVWY")[i % 3]
        text, pats = workloads.tiny_case(rng, alph, max_n=5000 if i % 10 == 0 else 300, max_p=12, max_len=24,
                                         other_frac=0.05 if i % 4 == 0 else 0.0)
        K = 1 + (i % 2) if len(pats) >= 2 else 1
        a = A.ac_build(pats, num_subsets=K, machine=A.AC_MACHINE_PFAC,
                       smem_table_bytes=64 if i % 5 == 0 else 0)
        same(A.ac_scan(a, text), oracle.scan(pats, text))
    w = workloads.config1()
    a = A.ac_build(w.patterns, alphabet="ACGT", machine=A.AC_MACHINE_PFAC)
    same(A.ac_scan(a, torch.from_numpy(w.text).cuda()), oracle.scan(w.patterns, w.text))
    w = workloads.config2(n=16 << 20)
    a = A.ac_build(w.patterns, alphabet="ACGT", machine=A.AC_MACHINE_PFAC)
    same(A.ac_scan(a, torch.from_numpy(w.text).cuda()), oracle.Machine(w.patterns).scan_mt(w.text, THREADS))
    with pytest.raises(A.AcError):
        A.ac_scan(a, torch.from_numpy(workloads.pack2(w.text)).cuda(), n=w.text.size, fmt=A.AC_PACKED2)


def test_failure_less_machine_config3():
    w = workloads.config3()
    a = A.ac_build(w.patterns, alphabet=w.alphabet, machine=A.AC_MACHINE_PFAC)
    same(A.ac_scan(a, torch.from_numpy(w.text).cuda()), oracle.Machine(w.patterns).scan_mt(w.text, THREADS))


def test_async_sort_paths():
    """Capacities at or below the single-launch rank sort's limit (8,192 keys) and above it (device radix sort)."""
    import itertools
    rng = np.random.default_rng(91)
    pats = [bytes(p) for p in itertools.product(b"ACGT", repeat=4)]   # every window matches
    a = A.ac_build(pats, alphabet="ACGT")
    for n in (5000, 8195, 60_000):
        text = workloads.dna_text(rng, n)
        want = oracle.scan(pats, text)
        M = want[0].shape[0]
        dt = torch.from_numpy(text).cuda()
        for cap in (M, M + 1, 8192, 1 << 17):
            if cap < M:
                continue
            d_m = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
            d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
            d_c = torch.zeros(len(pats), dtype=torch.int64, device="cuda")
            A.ac_scan_async(a, dt, n, A.AC_U8, None, d_m, cap, d_num, d_c)
            torch.cuda.synchronize()
            assert int(d_num.item()) == M
            got = d_m.view(-1, 2)[:M].cpu().numpy().view(np.uint32)
            same((got, d_c.cpu().numpy().view(np.uint64)), want)


def test_sort_of_keys_at_an_8_byte_offset():
    """The rank sort reads keys 16 bytes at a time when it can; a key buffer
    that starts 8 bytes past a 16-byte boundary takes its plain loads."""
    import itertools
    rng = np.random.default_rng(92)
    pats = [bytes(p) for p in itertools.product(b"ACGT", repeat=4)]
    a = A.ac_build(pats, alphabet="ACGT")
    for n in (3001, 6000):
        text = workloads.dna_text(rng, n)
        want = oracle.scan(pats, text)
        M = want[0].shape[0]
        cap = 8192
        dt = torch.from_numpy(text).cuda()
        keys = torch.zeros(cap + 1, dtype=torch.int64, device="cuda")[1:]
        d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
        d_c = torch.zeros(len(pats), dtype=torch.int64, device="cuda")
        A.ac_scan_keys_async(a, dt, n, A.AC_U8, None, keys, cap, d_num, d_c)
        d_m = torch.zeros(2 * cap, dtype=torch.int32, device="cuda")
        d_num2 = torch.zeros(1, dtype=torch.int64, device="cuda")
        A.ac_sort_keys_async(a, n, keys, d_num, cap, None, d_m, d_num2)
        torch.cuda.synchronize()
        assert int(d_num2.item()) == M
        got = d_m.view(-1, 2)[:M].cpu().numpy().view(np.uint32)
        same((got, d_c.cpu().numpy().view(np.uint64)), want)


def test_tune_and_table_caps():
    """ac_tune picks a configuration by timing; every shared-memory table cap
    (down to none) and the tuned configuration give the oracle's result."""
    w = workloads.config3(n=8 << 20, P=20_000)
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    a = A.ac_build(w.patterns, alphabet=w.alphabet)
    d = torch.from_numpy(w.text).cuda()
    for cap in (0, 64 << 10, 16 << 10, 4 << 10, 64):
        A.ac_set_scan_config(a, smem_table_bytes=cap)
        same(A.ac_scan(a, d), want)
    A.ac_set_scan_config(a)
    chosen = A.ac_tune(a, d)
    assert chosen["threads"] in (256, 512) and chosen["chains"] in (1, 2, 4)
    assert A.ac_get_scan_config(a) == chosen
    same(A.ac_scan(a, d), want)


@pytest.mark.parametrize("cap", [64, 1024, 16 << 10])
def test_optimistic_placement_repairs(cap):
    """AC_PLACE_OPT with a small power-of-two prefix: many stages reach a
    state beyond it and are walked again; the result stays exact. Chains = 1
    has no optimistic kernel and runs the hybrid one."""
    rng = np.random.default_rng(700 + cap)
    for i in range(60):
        alph = (b"ACGT", b"ab", b"ACDEFGHIKLMNPQRSTVWY")[i % 3]
        text, pats = workloads.tiny_case(rng, alph, max_n=3000, max_p=40, max_len=16,
                                         other_frac=0.03 if i % 4 == 0 else 0.0)
        K = 1 + (i % 3) if len(pats) >= 3 else 1
        a = A.ac_build(pats, num_subsets=K, placement=A.AC_PLACE_OPT, smem_table_bytes=cap, stride=1)
        A.ac_set_scan_config(a, **[dict(row_len=64, threads=64, chains=2, stage_bytes=16),
                                   dict(row_len=128, threads=128, chains=4),
                                   dict(row_len=96, threads=64, chains=1)][i % 3])
        want = oracle.scan(pats, text)
        same(A.ac_scan(a, text), want)
        if alph == b"ACGT" and not np.any(~np.isin(text, np.frombuffer(b"ACGT", np.uint8))) and a_is_acgt(pats):
            same(A.ac_scan(a, workloads.pack2(text), n=text.size, fmt=A.AC_PACKED2), want)


def a_is_acgt(pats):
    return set(b"".join(pats)) == set(b"ACGT")


def test_optimistic_placement_chosen_for_many_subsets():
    """Config 2 at 16 subsets: the automatic placement reads a power-of-two
    prefix optimistically; the same result as the hybrid placement."""
    w = workloads.config2(n=8 << 20)
    want = oracle.Machine(w.patterns).scan_mt(w.text, THREADS)
    d = torch.from_numpy(w.text).cuda()
    for placement in (A.AC_PLACE_AUTO, A.AC_PLACE_OPT, A.AC_PLACE_HYBRID):
        a = A.ac_build(w.patterns, alphabet="ACGT", num_subsets=16, placement=placement)
        for cfg in (dict(stride=1), dict(stride=1, stage_bytes=32), dict(stride=1, chains=4)):
            A.ac_set_scan_config(a, **cfg)
            same(A.ac_scan(a, d), want)
