"""The synthetic inputs (CPU only): each generator produces the shapes the
measured configurations state -- text sizes and alphabets, pattern counts,
length ranges, distinctness, the share of patterns cut from the text,
letter skew, batch and request-length laws, 2-bit packing -- so that a
measured number is a number on the stated workload. Reduced sizes where the
generator takes them as parameters (the laws do not depend on them).
"""
import os

import numpy as np

import oracle
import workloads as W

THREADS = os.cpu_count() or 4

DNA = np.frombuffer(W.DNA, np.uint8)
PROT = np.frombuffer(W.PROTEIN, np.uint8)


def check_patterns(pats, P, lo, hi, letters):
    assert len(pats) == P and len(set(pats)) == P          # exactly P, distinct
    lens = np.array([len(p) for p in pats])
    assert lens.min() >= lo and lens.max() <= hi
    assert lens.min() <= lo + 2 and lens.max() >= hi - 2    # the whole range is used
    allowed = set(letters.tolist())
    assert all(set(p) <= allowed for p in pats)


def cut_share(pats, text):
    """Share of the patterns that occur in the text (counted by the oracle)."""
    counts = oracle.Machine(pats).scan_mt(text, THREADS)[1]
    return float(np.mean(counts > 0))


def test_config1_shape():
    w = W.config1()
    assert w.text.size == 1 << 20 and set(np.unique(w.text)) <= set(DNA.tolist())
    check_patterns(w.patterns, 100, 8, 32, DNA)
    assert 0.45 <= cut_share(w.patterns, w.text) <= 0.6     # half cut from the text (random ones rarely occur)
    # uniform letters
    f = np.bincount(w.text, minlength=256)[DNA] / w.text.size
    assert np.all(np.abs(f - 0.25) < 0.01)


def test_config2_shape_at_reduced_size():
    w = W.config2(n=4 << 20)
    assert w.text.size == 4 << 20
    check_patterns(w.patterns, 10_000, 16, 64, DNA)
    assert 0.45 <= cut_share(w.patterns, w.text) <= 0.55


def test_config3_shape_at_reduced_size():
    w = W.config3(n=2 << 20, P=5_000)
    check_patterns(w.patterns, 5_000, 6, 20, PROT)
    assert 0.65 <= cut_share(w.patterns, w.text) <= 0.8      # 70% cut (short random ones may occur too)
    # Zipf 0.5 over a seeded letter order: frequency of rank k proportional to k^-0.5
    letters, probs = w.meta["letters"], w.meta["probs"]
    f = np.bincount(w.text, minlength=256)[np.frombuffer(letters, np.uint8)] / w.text.size
    want = np.arange(1, 21) ** -0.5
    assert np.allclose(f, want / want.sum(), atol=0.002) and np.allclose(probs, want / want.sum())


def test_config4_shape_reduced():
    w = W.config4(num_texts=300, hi=256 << 10, set_hi=8_000)
    lens = np.array([t.size for t in w.texts])
    assert lens.min() >= 1024 and lens.max() <= 256 << 10
    # log-uniform: log-lengths spread evenly over [ln 1 KiB, ln 256 KiB]
    q = np.quantile(np.log(lens), [0.25, 0.5, 0.75])
    lo, hi = np.log(1024), np.log(256 << 10)
    assert np.allclose(q, lo + (hi - lo) * np.array([0.25, 0.5, 0.75]), atol=0.5)
    assert set(np.unique(w.set_of_text)) <= set(range(8))
    sizes = w.meta["set_sizes"]
    assert sizes[0] == 1000 and sizes[-1] == 8_000 and sizes == sorted(sizes)
    for P, pats in zip(sizes, w.pattern_sets):
        check_patterns(pats, P, 12, 40, DNA)


def test_config5_sets_and_request_law():
    w = W.config5_sets(dna_P=500, prot_P=2_000, seed_text_len=1 << 20)
    assert len(w.pattern_sets) == 16
    for k, pats in enumerate(w.pattern_sets):
        if k < 8:
            check_patterns(pats, 500, 12, 40, DNA)
        else:
            check_patterns(pats, 2_000, 6, 20, PROT)
    rng = np.random.default_rng(1)
    t, sets, lens = W.request_stream(rng, 1000.0, 20_000)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1e-3) < 5e-5                     # Poisson arrivals at the offered rate
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.05        # exponential gaps
    assert set(np.unique(sets)) == set(range(16))
    assert lens.min() >= 4096 and lens.max() <= 64 << 20
    assert abs(np.median(np.log(lens)) - 0.5 * (np.log(4096) + np.log(64 << 20))) < 0.2


def test_pack2_round_trip_and_layout():
    rng = np.random.default_rng(2)
    for n in (0, 1, 3, 4, 5, 1000, 4097):
        t = W.dna_text(rng, n)
        p = W.pack2(t)
        assert p.size == (n + 3) // 4
        assert np.array_equal(W.unpack2(p, n), t)
    # symbol 4i + j in bits [2j, 2j + 2) of byte i, A C G T = 0 1 2 3
    assert W.pack2(np.frombuffer(b"ACGTTGCA", np.uint8)).tolist() == [0b11100100, 0b00011011]
