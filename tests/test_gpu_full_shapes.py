"""GPU parity at the shapes the benchmark times, element by element.

* Config 4 at full size: 4,096 DNA texts of log-uniform length in
  [1 KiB, 4 MiB] (about 2.1 GB) against 8 resident pattern sets of 1,000 to
  50,000 patterns of U[12,40] letters, through both batch paths with the
  flags the benchmark uses: texts one automaton at a time as one text (the
  default), and the one-launch arena kept as a plan and replayed as a CUDA
  graph (first call plans and autotunes, later calls replay). A sample of
  texts also goes through one ac_scan_async call per text (the per-call
  arm).
* Config 5's 16 sets at their stated sizes (8 DNA sets of 5,000 patterns of
  U[12,40], 8 protein sets of 20,000 patterns of U[6,20]) with requests of
  log-uniform length in [4 KiB, 64 MiB] (both ends included): each request
  scanned alone equals the same request served in the mix, which equals the
  oracle.
* The shapes of the paper's Section V (Figs. 7-8): 0.5 M and 1.5 M random DNA
  patterns of 15 to 25 letters (10 and 30 MB of patterns) against 70 KB and
  100 KB texts with 50 embedded occurrences; the folded machine built on the
  host and on the GPU, and the failure-less machine (Section II.B).

Every result is compared with the oracle (failure-link Aho-Corasick of
Section II.A, plain C) on the same seeded inputs: the sorted (end position,
pattern id) list and the per-pattern counts.
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import workloads
from paper_1403_1305_gb300 import ac as A

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CORES = os.cpu_count() or 4


@pytest.fixture(scope="module", autouse=True)
def cuda_device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    yield
    A.ac_batch_release()


def oracle_results(machines, jobs):
    """Oracle result of every (machine index, text) job: texts scanned in
    parallel on the host cores (the oracle machine is read-only during a
    scan), long texts over chunks on all cores."""
    out = [None] * len(jobs)

    def one(i):
        k, t = jobs[i]
        out[i] = machines[k].scan_mt(t, CORES) if t.size > (16 << 20) else machines[k].scan(t)

    order = sorted(range(len(jobs)), key=lambda i: -jobs[i][1].size)
    big = [i for i in order if jobs[i][1].size > (16 << 20)]
    for i in big:
        one(i)
    with cf.ThreadPoolExecutor(CORES) as ex:
        list(ex.map(one, [i for i in order if jobs[i][1].size <= (16 << 20)]))
    return out


def assert_same(got, want, counts=True, what=""):
    assert len(got) == len(want)
    for i, ((m, c), (wm, wc)) in enumerate(zip(got, want)):
        assert np.array_equal(m, wm), f"{what}: matches of item {i} differ"
        if counts:
            assert np.array_equal(c, wc), f"{what}: counts of item {i} differ"
        else:
            assert c is None


@pytest.fixture(scope="module")
def config4():
    w = workloads.config4()
    assert len(w.texts) == 4096 and w.meta["set_sizes"][0] == 1000 and w.meta["set_sizes"][-1] == 50_000
    machines = [oracle.Machine(s) for s in w.pattern_sets]
    want = oracle_results(machines, [(int(a), t) for a, t in zip(w.set_of_text, w.texts)])
    autos = [A.ac_build(s, alphabet="ACGT") for s in w.pattern_sets]
    d_texts = [torch.from_numpy(t).cuda() for t in w.texts]
    items = [(int(a), d, t.size, A.AC_U8) for a, d, t in zip(w.set_of_text, d_texts, w.texts)]
    torch.cuda.synchronize()
    return w, autos, items, want


def test_config4_one_text_per_automaton(config4):
    w, autos, items, want = config4
    got = A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=A.AC_BATCH_NO_COUNTS)
    assert_same(got, want, counts=False, what="one text per automaton, no counts")
    got = A.ac_scan_batch(autos, items, mem=A.AC_DEVICE)
    assert_same(got, want, what="one text per automaton, counts")


def test_config4_one_launch_graph(config4):
    w, autos, items, want = config4
    fl = A.AC_BATCH_GRAPH | A.AC_BATCH_NO_COUNTS
    for rep in range(3):  # plan + autotune, then graph replays
        got = A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=fl)
        assert_same(got, want, counts=False, what=f"one-launch graph, call {rep}")
    got = A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=A.AC_BATCH_GRAPH)
    assert_same(got, want, what="one-launch graph with counts")
    A.ac_batch_release()


def test_config4_per_call_sample(config4):
    """The per-call arm (ac_scan_async per text) on every 32nd text."""
    w, autos, items, want = config4
    stream = torch.cuda.Stream()
    for i in range(0, len(items), 32):
        ai, d, n, f = items[i]
        a = autos[ai]
        cap = max(4096, n // 256)
        d_m = torch.empty(cap, dtype=torch.int64, device="cuda")
        d_num = torch.zeros(1, dtype=torch.int64, device="cuda")
        d_c = torch.empty(a.num_patterns, dtype=torch.int64, device="cuda")
        with torch.cuda.stream(stream):
            A.ac_scan_async(a, d, n, f, stream, d_m, cap, d_num, d_c)
        stream.synchronize()
        M = int(d_num.item())
        wm, wc = want[i]
        assert M == wm.shape[0]
        got = d_m[:M].cpu().numpy().view(np.uint32).reshape(M, 2)
        assert np.array_equal(got, wm)
        assert np.array_equal(d_c.cpu().numpy().view(np.uint64), wc)


@pytest.fixture(scope="module")
def config5():
    w = workloads.config5_sets()
    assert [len(s) for s in w.pattern_sets] == [5000] * 8 + [20_000] * 8
    autos = [A.ac_build(s, alphabet=a) for s, a in zip(w.pattern_sets, w.set_alphabet)]
    machines = [oracle.Machine(s) for s in w.pattern_sets]
    rng = np.random.default_rng(1056)
    _, sets, lens = workloads.request_stream(rng, 1000.0, 40)
    lens = list(lens) + [4096, 64 << 20, 4096, 64 << 20]
    sets = list(sets) + [0, 1, 8, 15]  # both ends of the length range, DNA and protein
    reqs = []
    for k, n in zip(sets, lens):
        letters, probs = w.set_letters[int(k)]
        reqs.append((int(k), workloads.iid_text(rng, int(n), letters, probs)))
    want = oracle_results(machines, reqs)
    return autos, reqs, want


@pytest.mark.parametrize("staging", [A.AC_STAGE_DEVICE, A.AC_STAGE_PINNED])
def test_config5_alone_mixed_oracle(config5, staging):
    autos, reqs, want = config5
    alone = [A.ac_scan(autos[k], t) for k, t in reqs]
    assert_same(alone, want, what="alone")
    srv = A.ac_serve_create(autos, num_streams=3, max_batch_items=64, max_wait_us=100,
                            device_mem_budget=8 << 30, staging=staging)
    tickets = [A.ac_serve_submit(srv, k, t) for k, t in reqs]
    mixed = [A.ac_serve_wait(srv, tk, 600_000) for tk in tickets]
    st = A.ac_serve_stats(srv)
    A.ac_serve_destroy(srv)
    assert st["submitted"] == st["completed"] == len(reqs)
    assert_same(mixed, want, what="served")


@pytest.mark.parametrize("P", [500_000, 1_500_000])
def test_paper_section5_shapes(P):
    rng = np.random.default_rng(1176)
    pats = workloads.random_patterns(rng, P, 15, 25, workloads.DNA)
    texts = [workloads.embed(rng, workloads.dna_text(rng, kb * 1000), pats, 50) for kb in (70, 100)]
    m = oracle.Machine(pats)
    want = [m.scan(t) for t in texts]
    for t, (wm, _) in zip(texts, want):
        assert wm.shape[0] >= 50  # the embedded occurrences are found
    del m
    for mk, bld in ((A.AC_MACHINE_DFA, A.AC_BUILDER_HOST), (A.AC_MACHINE_DFA, A.AC_BUILDER_DEVICE),
                    (A.AC_MACHINE_PFAC, A.AC_BUILDER_HOST)):
        a = A.ac_build(pats, alphabet="ACGT", machine=mk, builder=bld)
        got = [A.ac_scan(a, t) for t in texts]
        assert_same(got, want, what=f"machine {mk} builder {bld}")
        dev = [torch.from_numpy(t).cuda() for t in texts]
        got = [A.ac_scan(a, d) for d in dev]
        assert_same(got, want, what=f"machine {mk} builder {bld}, device text")
        del a
