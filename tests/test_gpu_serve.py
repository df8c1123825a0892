"""GPU tests of the serving loop (ac_serve_*).

The same requests are scanned alone (ac_scan) and submitted together to a
server that coalesces them into batched launches on several streams; every
result must be identical in both cases and equal to the oracle. Also checked:
texts staged in device memory or in the pinned slab, and batches that mix
both (the device share of the budget spent); poll/wait semantics, refusal
when the queue is full or a text exceeds the memory budget, an unknown
staging mode, and a server destroyed with requests still queued.
"""
import numpy as np
import pytest

import oracle
import workloads
from paper_1403_1305_gb300 import ac as A

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def fleet():
    """4 DNA and 4 protein pattern sets (config-5 shape, fewer and smaller)."""
    rng = np.random.default_rng(51)
    sets, alph, kinds, texts = [], [], [], []
    dna_l = np.frombuffer(b"ACGT", np.uint8)
    for _ in range(4):
        src = workloads.dna_text(rng, 1 << 20)
        sets.append(workloads.draw_patterns(rng, src, 500, 12, 40, 0.5, dna_l))
        alph.append(workloads.DNA)
        kinds.append((dna_l, None))
    for _ in range(4):
        letters, probs = workloads.zipf_letters(rng)
        src = workloads.iid_text(rng, 1 << 20, letters, probs)
        sets.append(workloads.draw_patterns(rng, src, 2000, 6, 20, 0.5, letters, probs))
        alph.append(workloads.PROTEIN)
        kinds.append((letters, probs))
    autos = [A.ac_build(s, alphabet=a) for s, a in zip(sets, alph)]
    return sets, autos, kinds, [oracle.Machine(s) for s in sets]


def requests(rng, kinds, count, lo=1 << 10, hi=1 << 20):
    out = []
    for _ in range(count):
        k = int(rng.integers(0, len(kinds)))
        n = int(workloads.log_uniform_lengths(rng, 1, lo, hi)[0])
        letters, probs = kinds[k]
        out.append((k, workloads.iid_text(rng, n, letters, probs)))
    return out


@pytest.mark.parametrize("streams,max_items,staging", [(1, 1, A.AC_STAGE_DEVICE), (2, 8, A.AC_STAGE_DEVICE),
                                                       (3, 256, A.AC_STAGE_DEVICE), (2, 8, A.AC_STAGE_PINNED)])
def test_alone_and_in_the_mix_are_identical(fleet, streams, max_items, staging):
    sets, autos, kinds, machines = fleet
    rng = np.random.default_rng(52 + streams)
    reqs = requests(rng, kinds, 60)
    alone = [A.ac_scan(autos[k], t) for k, t in reqs]
    srv = A.ac_serve_create(autos, num_streams=streams, max_batch_items=max_items, max_wait_us=200,
                            staging=staging)
    tickets = [A.ac_serve_submit(srv, k, t) for k, t in reqs]
    mixed = [A.ac_serve_wait(srv, tk, 120_000) for tk in tickets]
    st = A.ac_serve_stats(srv)
    A.ac_serve_destroy(srv)
    assert st["submitted"] == st["completed"] == len(reqs)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for (k, t), (am, ac), (mm, mc) in zip(reqs, alone, mixed):
        assert np.array_equal(am, mm) and np.array_equal(ac, mc)
        wm, wc = machines[k].scan(t)
        assert np.array_equal(mm, wm) and np.array_equal(mc, wc)


def test_poll_wait_and_tickets(fleet):
    sets, autos, kinds, machines = fleet
    rng = np.random.default_rng(60)
    srv = A.ac_serve_create(autos, num_streams=1)
    big = workloads.dna_text(rng, 32 << 20)
    tk = A.ac_serve_submit(srv, 0, big)
    with pytest.raises(A.AcError) as e:          # not done within 0 ms
        A.ac_serve_wait(srv, tk, 0)
    assert e.value.code == A.AC_ETIMEDOUT
    got = None
    while got is None:
        got = A.ac_serve_poll(srv, tk)
    wm, wc = machines[0].scan(big)
    assert np.array_equal(got[0], wm) and np.array_equal(got[1], wc)
    with pytest.raises(A.AcError) as e:          # consumed
        A.ac_serve_poll(srv, tk)
    assert e.value.code == A.AC_EINVAL
    with pytest.raises(A.AcError) as e:          # never issued
        A.ac_serve_wait(srv, 10 ** 9, 10)
    assert e.value.code == A.AC_EINVAL
    A.ac_serve_destroy(srv)


def test_queue_full_and_budget(fleet):
    sets, autos, kinds, machines = fleet
    rng = np.random.default_rng(61)
    srv = A.ac_serve_create(autos, num_streams=1, max_queue=3, max_batch_items=1)
    big = workloads.dna_text(rng, 64 << 20)
    small = workloads.dna_text(rng, 5000)
    tickets, refused = [A.ac_serve_submit(srv, 0, big)], 0
    for _ in range(6):
        try:
            tickets.append(A.ac_serve_submit(srv, 1, small))
        except A.AcError as e:
            assert e.code == A.AC_EBUSY
            refused += 1
    assert refused >= 1
    for tk in tickets:
        A.ac_serve_wait(srv, tk, 120_000)
    A.ac_serve_destroy(srv)
    srv = A.ac_serve_create(autos, device_mem_budget=1 << 20)
    with pytest.raises(A.AcError) as e:
        A.ac_serve_submit(srv, 0, big)
    assert e.value.code == A.AC_ERANGE
    A.ac_serve_destroy(srv)


def test_destroy_with_queued_requests(fleet):
    sets, autos, kinds, machines = fleet
    rng = np.random.default_rng(62)
    srv = A.ac_serve_create(autos, num_streams=2)
    for k, t in requests(rng, kinds, 20):
        A.ac_serve_submit(srv, k, t)
    A.ac_serve_destroy(srv)          # drains the queue and returns


def test_device_staging_overflows_to_the_slab(fleet):
    """A 6 MiB budget holds a few 1 MiB texts in device memory at a time; the
    rest wait in the pinned slab, so batches mix both kinds."""
    sets, autos, kinds, machines = fleet
    rng = np.random.default_rng(63)
    reqs = requests(rng, kinds, 40, lo=(1 << 20) - 4096, hi=1 << 20)
    srv = A.ac_serve_create(autos, num_streams=2, max_batch_items=16, max_wait_us=2000,
                            device_mem_budget=6 << 20)
    tickets = [A.ac_serve_submit(srv, k, t) for k, t in reqs]
    got = [A.ac_serve_wait(srv, tk, 120_000) for tk in tickets]
    A.ac_serve_destroy(srv)
    for (k, t), (m, c) in zip(reqs, got):
        wm, wc = machines[k].scan(t)
        assert np.array_equal(m, wm) and np.array_equal(c, wc)


def test_unknown_staging(fleet):
    sets, autos, kinds, machines = fleet
    with pytest.raises(A.AcError) as e:
        A.ac_serve_create(autos, staging=2)
    assert e.value.code == A.AC_EINVAL


def test_latency_counts_from_the_given_arrival(fleet):
    """ac_serve_submit_at: a request that arrived 200 ms before it was
    submitted is at least 200 ms late in the server's percentiles, and its
    result is the same."""
    import time
    sets, autos, kinds, machines = fleet
    rng = np.random.default_rng(64)
    reqs = requests(rng, kinds, 8, lo=4096, hi=1 << 16)
    srv = A.ac_serve_create(autos, num_streams=1)
    past = time.monotonic_ns() - 200_000_000
    tickets = [A.ac_serve_submit_at(srv, k, t, past) for k, t in reqs]
    got = [A.ac_serve_wait(srv, tk, 60_000) for tk in tickets]
    st = A.ac_serve_stats(srv)
    A.ac_serve_destroy(srv)
    assert st["p50_ms"] >= 200.0 and st["p99_ms"] < 60_000
    for (k, t), (m, c) in zip(reqs, got):
        wm, wc = machines[k].scan(t)
        assert np.array_equal(m, wm) and np.array_equal(c, wc)
