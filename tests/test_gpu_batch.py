"""GPU parity of ac_scan_batch: every item of a batch against the oracle.

Batches mix automata (several pattern sets, subset counts), alphabets (DNA
and protein, which go to separate launches), text formats, empty and short
texts, and memory kinds, through both batch paths (byte texts one
automaton at a time as one text, separated by a byte outside the alphabet;
the one-launch arena); the graph-replay plan is checked on repeat calls,
including after the texts change in place.
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
    yield
    A.ac_batch_release()


def check(results, items, pattern_sets, texts_np, counts=True):
    assert len(results) == len(items)
    machines = [oracle.Machine(ps) for ps in pattern_sets]
    for (m, c), (ai, _t, n, fmt), txt in zip(results, items, texts_np):
        want_m, want_c = machines[ai].scan(txt)
        assert np.array_equal(m, want_m)
        if counts:
            assert np.array_equal(c, want_c)
        else:
            assert c is None


def make_sets(rng, texts, sizes, lo, hi):
    return [workloads.draw_patterns(rng, texts, P, lo, hi, 0.5, np.frombuffer(b"ACGT", np.uint8)) for P in sizes]


def test_mixed_batch_host_and_device():
    rng = np.random.default_rng(41)
    lens = [0, 1, 15, 16, 17, 63, 64, 65, 1000, 4097, 20_000, 70_001] + list(
        workloads.log_uniform_lengths(rng, 40, 100, 200_000))
    texts = [workloads.dna_text(rng, int(n)) for n in lens]
    sets = make_sets(rng, [t for t in texts if len(t) > 100], [30, 300, 1200], 4, 30)
    autos = [A.ac_build(sets[0], alphabet="ACGT"), A.ac_build(sets[1], alphabet="ACGT", num_subsets=3),
             A.ac_build(sets[2], alphabet="ACGT")]
    ai = rng.integers(0, 3, size=len(texts))
    items = [(int(a), t, t.size, A.AC_U8) for a, t in zip(ai, texts)]
    check(A.ac_scan_batch(autos, items), items, sets, texts)
    check(A.ac_scan_batch(autos, items, flags=A.AC_BATCH_NO_COUNTS), items, sets, texts, counts=False)
    dev = [(a, torch.from_numpy(t).cuda() if t.size else torch.zeros(1, dtype=torch.uint8, device="cuda"), n, f)
           for a, t, n, f in items]
    check(A.ac_scan_batch(autos, dev, mem=A.AC_DEVICE), items, sets, texts)
    # the one-launch arena (texts one automaton at a time as one text is the default for byte texts)
    check(A.ac_scan_batch(autos, items, flags=A.AC_BATCH_ONE_LAUNCH), items, sets, texts)
    check(A.ac_scan_batch(autos, dev, mem=A.AC_DEVICE, flags=A.AC_BATCH_ONE_LAUNCH | A.AC_BATCH_NO_COUNTS),
          items, sets, texts, counts=False)


def test_packed_and_protein_classes_in_one_call():
    rng = np.random.default_rng(42)
    dna = [workloads.dna_text(rng, int(n)) for n in (5000, 777, 123_457)]
    letters, probs = workloads.zipf_letters(rng)
    prot = [workloads.iid_text(rng, int(n), letters, probs) for n in (9000, 31)]
    dset = workloads.draw_patterns(rng, dna, 200, 6, 24, 0.6, np.frombuffer(b"ACGT", np.uint8))
    pset = workloads.draw_patterns(rng, prot[:1], 300, 3, 10, 0.6, letters, probs)
    autos = [A.ac_build(dset, alphabet="ACGT"), A.ac_build(pset, alphabet=workloads.PROTEIN)]
    items = [(0, workloads.pack2(dna[0]), dna[0].size, A.AC_PACKED2), (1, prot[0], prot[0].size, A.AC_U8),
             (0, dna[1], dna[1].size, A.AC_U8), (1, prot[1], prot[1].size, A.AC_U8),
             (0, workloads.pack2(dna[2]), dna[2].size, A.AC_PACKED2)]
    texts = [dna[0], prot[0], dna[1], prot[1], dna[2]]
    check(A.ac_scan_batch(autos, items), items, [dset, pset], texts)


def test_graph_plan_replay_and_in_place_change():
    rng = np.random.default_rng(43)
    texts = [workloads.dna_text(rng, int(n)) for n in workloads.log_uniform_lengths(rng, 64, 1024, 300_000)]
    sets = make_sets(rng, texts, [500, 2000], 8, 32)
    autos = [A.ac_build(s, alphabet="ACGT") for s in sets]
    dev = [torch.from_numpy(t).cuda() for t in texts]
    ai = rng.integers(0, 2, size=len(texts))
    items = [(int(a), d, t.size, A.AC_U8) for a, d, t in zip(ai, dev, texts)]
    for _ in range(3):  # plan + autotune, then graph replays
        check(A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=A.AC_BATCH_GRAPH), items, sets, texts)
    # same pointers, new contents (more matches: patterns written into the texts)
    for d, t in zip(dev, texts):
        for p in sets[0][:50]:
            if t.size > 2 * len(p):
                o = int(rng.integers(0, t.size - len(p)))
                t[o:o + len(p)] = np.frombuffer(p, np.uint8)
        d.copy_(torch.from_numpy(t).cuda())
    torch.cuda.synchronize()
    check(A.ac_scan_batch(autos, items, mem=A.AC_DEVICE, flags=A.AC_BATCH_GRAPH), items, sets, texts)
    # host texts through a graph plan
    hitems = [(a, t, n, f) for (a, _d, n, f), t in zip(items, texts)]
    for _ in range(2):
        check(A.ac_scan_batch(autos, hitems, flags=A.AC_BATCH_GRAPH), hitems, sets, texts)
    A.ac_batch_release()


def test_config4_shape_reduced():
    """Config-4 shape at reduced size: 256 texts of log-uniform length in
    [1 KiB, 256 KiB] against 8 pattern sets of 1,000..20,000 patterns U[12,40]."""
    w = workloads.config4(num_texts=256, hi=256 << 10, set_hi=20_000)
    autos = [A.ac_build(s, alphabet="ACGT") for s in w.pattern_sets]
    items = [(int(a), t, t.size, A.AC_U8) for a, t in zip(w.set_of_text, w.texts)]
    res = A.ac_scan_batch(autos, items)
    check(res, items, w.pattern_sets, w.texts)
    dev = [(a, torch.from_numpy(t).cuda(), n, f) for a, t, n, f in items]
    check(A.ac_scan_batch(autos, dev, mem=A.AC_DEVICE), items, w.pattern_sets, w.texts)
    check(A.ac_scan_batch(autos, dev, mem=A.AC_DEVICE, flags=A.AC_BATCH_ONE_LAUNCH), items, w.pattern_sets, w.texts)


def test_separator_bytes_inside_texts():
    """Texts one automaton at a time: bytes outside the alphabet inside the
    texts, texts that end or start with them, and device texts at odd
    offsets (not 16-byte aligned) in the gather."""
    rng = np.random.default_rng(43)
    clean = [workloads.dna_text(rng, n).copy() for n in (1, 2, 17, 33, 300, 5000, 70_000, 250_001)]
    sets = make_sets(rng, [t for t in clean if len(t) > 100], [50, 400], 3, 20)
    texts = []
    for t in clean:
        t = t.copy()
        mask = rng.random(t.size) < 0.02
        t[mask] = rng.choice(np.frombuffer(b"N\x00xACGT", np.uint8), size=int(mask.sum()))
        if t.size > 2:
            t[0], t[-1] = ord("N"), 0
        texts.append(t)
    autos = [A.ac_build(sets[0], alphabet="ACGT"), A.ac_build(sets[1], alphabet="ACGT")]
    items = [(i % 2, t, t.size, A.AC_U8) for i, t in enumerate(texts)]
    check(A.ac_scan_batch(autos, items), items, sets, texts)
    big = torch.zeros(sum(t.size + 3 for t in texts) + 64, dtype=torch.uint8, device="cuda")
    dev, at = [], 5
    for (a, t, n, f) in items:
        big[at:at + n] = torch.from_numpy(t).cuda()
        dev.append((a, big[at:at + n], n, f))
        at += n + 3
    check(A.ac_scan_batch(autos, dev, mem=A.AC_DEVICE), items, sets, texts)


def test_batch_errors():
    a = A.ac_build([b"ACGT"], alphabet="ACGT")
    with pytest.raises(A.AcError) as e:
        A.ac_scan_batch([a], [(1, b"ACGT", 4, A.AC_U8)])
    assert e.value.code == A.AC_EINVAL
    b = A.ac_build([b"AB", b"C"])
    with pytest.raises(A.AcError) as e:
        A.ac_scan_batch([b], [(0, b"\x00", 4, A.AC_PACKED2)])
    assert e.value.code == A.AC_EINVAL


def test_flat_results():
    """flat=True: one matches array with per-text offsets, the same records
    as the per-text pairs."""
    rng = np.random.default_rng(44)
    texts = [workloads.dna_text(rng, int(n)) for n in (0, 5, 3000, 70_000, 1)]
    sets = make_sets(rng, [t for t in texts if t.size > 100], [80, 400], 4, 20)
    autos = [A.ac_build(s, alphabet="ACGT") for s in sets]
    items = [(i % 2, t, t.size, A.AC_U8) for i, t in enumerate(texts)]
    pairs = A.ac_scan_batch(autos, items)
    m, mo, c, co = A.ac_scan_batch(autos, items, flat=True)
    assert mo.shape == (len(items) + 1,) and co.shape == (len(items) + 1,)
    for i, (pm, pc) in enumerate(pairs):
        assert np.array_equal(m[mo[i]:mo[i + 1]], pm)
        assert np.array_equal(c[co[i]:co[i + 1]], pc)
    m2, mo2, c2, co2 = A.ac_scan_batch(autos, items, flags=A.AC_BATCH_NO_COUNTS, flat=True)
    assert np.array_equal(m2, m) and np.array_equal(mo2, mo) and c2 is None and co2 is None
