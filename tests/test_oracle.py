"""Pins for the oracle (CPU only).

The oracle is checked against things other than itself:
  * the paper's worked examples with the state numbers its text quotes
    (Section II.A / Fig. 1, Section II.B / Fig. 4, Section IV.A / Fig. 6),
  * the definition of the result set (brute force) on thousands of random
    small cases, and the failure-less walk of Section II.B on the same cases,
  * a closed form: all k-mers as the pattern set match every window, so the
    counts are the k-mer histogram (computed here with numpy, not the oracle),
  * the input-focused chunked scan (Section III) equals the whole scan, and
    texts joined by bytes outside the alphabet scan as each text alone,
  * planted mistakes: compiling ``ac_oracle.c`` with ``-DORACLE_MUTANT=k``
    gives variants with a plausible bug each, and every one of them must fail
    at least one of the pins above.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- pin checks
# Each returns a list of failure descriptions (empty = pass), so the same
# checks can be run against a mutant build.

def check_fig1(lib):
    g = load_golden("fig1_abede.json")
    errs = []
    m = oracle.Machine(g["patterns"], True, lib)
    matches, counts = m.scan(g["text"])
    if matches.tolist() != g["matches"]:
        errs.append(f"fig1 matches {matches.tolist()}")
    if counts.tolist() != g["counts"]:
        errs.append(f"fig1 counts {counts.tolist()}")
    for prefix, sid in g["states_quoted"].items():
        if m.state_of(prefix) != sid:
            errs.append(f"fig1 state of {prefix} = {m.state_of(prefix)}")
    for s, f in g["failure_quoted"].items():
        if m.fail(m.state_of(s)) != m.state_of(f):
            errs.append(f"fig1 f({s})")
    tr = m.trace(g["text"]).tolist()
    for got, want in zip(tr, g["trace_quoted"]):
        if want is not None and got != want:
            errs.append(f"fig1 trace {tr}")
            break
    return errs


def check_fig4(lib):
    g = load_golden("fig4_pfac_abede.json")
    errs = []
    m = oracle.Machine(g["patterns"], False, lib)
    for start, walk in g["walks_quoted"].items():
        got = m.pfac_walk(g["text"], int(start))
        if got != walk:
            errs.append(f"fig4 walk from {start}: {got}")
    matches, _ = m.pfac(g["text"])
    if matches.tolist() != g["matches"]:
        errs.append(f"fig4 matches {matches.tolist()}")
    return errs


def check_fig6(lib):
    g = load_golden("fig6_ushers.json")
    errs = []
    for wf in (True, False):
        m = oracle.Machine(g["patterns"], wf, lib)
        matches, counts = m.scan(g["text"]) if wf else m.pfac(g["text"])
        if matches.tolist() != g["matches"]:
            errs.append(f"fig6 matches (failure={wf}) {matches.tolist()}")
        if counts.tolist() != g["counts"]:
            errs.append(f"fig6 counts (failure={wf}) {counts.tolist()}")
        for prefix, sid in g["states_quoted"].items():
            if m.state_of(prefix) != sid:
                errs.append(f"fig6 state of {prefix}")
        if not wf:
            for start, walk in g["walks_quoted"].items():
                got = m.pfac_walk(g["text"], int(start))
                if len(got) != len(walk) or any(w is not None and w != x for w, x in zip(walk, got)):
                    errs.append(f"fig6 walk from {start}: {got}")
    return errs


def check_random(lib, cases=400, seed=7, alphabets=(b"ab", b"ACGT")):
    """AC scan == PFAC == brute force == chunked scan on random small cases."""
    errs = []
    rng = np.random.default_rng(seed)
    for i in range(cases):
        alph = alphabets[i % len(alphabets)]
        text, pats = workloads.tiny_case(rng, alph, max_n=48, max_p=7, max_len=5,
                                         other_frac=0.1 if i % 3 == 0 else 0.0)
        want, wc = oracle.brute(pats, text, lib)
        got, gc = oracle.Machine(pats, True, lib).scan(text)
        if not np.array_equal(got, want) or not np.array_equal(gc, wc):
            errs.append(f"random case {i}: scan != brute")
            break
        got, _ = oracle.Machine(pats, False, lib).pfac(text)
        if not np.array_equal(got, want):
            errs.append(f"random case {i}: pfac != brute")
            break
    return errs


def kmer_ids(text, k, letters):
    """Expected (end, id) for the all-k-mers pattern set, computed with numpy:
    id = base-sigma number of the window (first letter most significant),
    windows holding a byte outside ``letters`` produce nothing."""
    lut = np.full(256, -1, dtype=np.int64)
    for i, b in enumerate(letters):
        lut[b] = i
    codes = lut[np.asarray(text, dtype=np.uint8)]
    if len(codes) < k:
        return np.zeros((0, 2), np.uint32)
    win = np.lib.stride_tricks.sliding_window_view(codes, k)
    ok = (win >= 0).all(axis=1)
    sigma = len(letters)
    ids = (win * (sigma ** np.arange(k - 1, -1, -1))).sum(axis=1)
    ends = np.arange(k - 1, len(codes))
    return np.stack([ends[ok], ids[ok]], axis=1).astype(np.uint32)


def check_kmers(lib, n=20000, seed=11):
    errs = []
    rng = np.random.default_rng(seed)
    for letters, k in ((workloads.DNA, 4), (workloads.PROTEIN, 2)):
        pats = [bytes(p) for p in itertools.product(letters, repeat=k)]
        text = workloads.iid_text(rng, n, np.frombuffer(letters, np.uint8))
        text[rng.random(n) < 0.01] = ord("N") if letters == workloads.DNA else ord("B")
        want = kmer_ids(text, k, letters)
        got, counts = oracle.Machine(pats, True, lib).scan(text)
        if not np.array_equal(got, want):
            errs.append(f"k-mers k={k}: matches differ")
        hist = np.bincount(want[:, 1].astype(np.int64), minlength=len(pats)).astype(np.uint64)
        if not np.array_equal(counts, hist):
            errs.append(f"k-mers k={k}: counts differ")
    return errs


ALL_CHECKS = (check_fig1, check_fig4, check_fig6, check_random, check_kmers)


# ---------------------------------------------------------------- tests

def test_fig1_worked_example():
    assert check_fig1(oracle.load()) == []


def test_fig4_pfac_worked_example():
    assert check_fig4(oracle.load()) == []


def test_fig6_worked_example():
    assert check_fig6(oracle.load()) == []


def test_random_small_cases_against_brute_force():
    assert check_random(oracle.load(), cases=6000, seed=1) == []


def test_random_cases_wide_alphabet():
    lib = oracle.load()
    rng = np.random.default_rng(3)
    for i in range(500):
        text, pats = workloads.tiny_case(rng, b"ACDEFGHIKL", max_n=200, max_p=20, max_len=4)
        assert np.array_equal(oracle.Machine(pats, True, lib).scan(text)[0], oracle.brute(pats, text, lib)[0])


def test_kmer_closed_form():
    assert check_kmers(oracle.load()) == []


def test_chunked_threads_equal_whole_scan():
    """Section III's input-focused split: chunks warmed up on (max length - 1)
    characters reproduce the single scan exactly, for any thread count."""
    lib = oracle.load()
    rng = np.random.default_rng(5)
    for i in range(200):
        text, pats = workloads.tiny_case(rng, b"ACGT", max_n=300, max_p=12, max_len=9)
        m = oracle.Machine(pats, True, lib)
        want = m.scan(text)[0]
        for t in (1, 2, 3, 7, 64):
            assert np.array_equal(m.scan_mt(text, t)[0], want), (i, t)


def test_texts_joined_by_a_byte_outside_the_alphabet():
    """The property one-text-per-automaton batches rest on (Section II.A: no
    pattern holds a byte outside the alphabet, so the walk returns to the
    root there): texts joined by one or more such bytes give exactly each
    text's own matches, shifted by the text's offset, and nothing else."""
    lib = oracle.load()
    rng = np.random.default_rng(8)
    for i in range(100):
        n_texts = int(rng.integers(1, 6))
        texts, pats = [], None
        for _ in range(n_texts):
            t, p = workloads.tiny_case(rng, b"ACGT", max_n=120, max_p=10, max_len=8)
            texts.append(t)
            pats = p if pats is None else pats + p
        m = oracle.Machine(pats, True, lib)
        joined, offs = [], []
        for t in texts:
            if joined:
                joined.append(np.full(int(rng.integers(1, 17)), ord("N") if i % 2 else 0, np.uint8))
            offs.append(sum(x.size for x in joined))
            joined.append(t)
        whole = np.concatenate(joined) if joined else np.zeros(0, np.uint8)
        got = m.scan(whole)[0]
        want = [np.asarray(m.scan(t)[0], np.int64) + np.array([o, 0]) for t, o in zip(texts, offs)]
        want = np.concatenate(want) if want else np.zeros((0, 2), np.int64)
        assert np.array_equal(np.asarray(got, np.int64), want), i


def test_edge_cases():
    lib = oracle.load()
    # empty text
    got, counts = oracle.scan([b"A"], b"", lib)
    assert got.shape == (0, 2) and counts.tolist() == [0]
    # pattern longer than the text
    assert oracle.scan([b"AAAA"], b"AAA", lib)[0].shape == (0, 2)
    # duplicates: every id is reported
    got, counts = oracle.scan([b"AC", b"AC", b"C"], b"ACAC", lib)
    assert got.tolist() == [[1, 0], [1, 1], [1, 2], [3, 0], [3, 1], [3, 2]]
    assert counts.tolist() == [2, 2, 2]
    # overlapping occurrences of one pattern
    got, _ = oracle.scan([b"AA"], b"AAAA", lib)
    assert got[:, 0].tolist() == [1, 2, 3]
    # out-of-alphabet bytes break matches
    assert oracle.scan([b"AC"], b"ANC", lib)[0].shape == (0, 2)
    # empty pattern and empty set are rejected
    with pytest.raises(ValueError):
        oracle.Machine([b"A", b""], True, lib)
    with pytest.raises(ValueError):
        oracle.Machine([], True, lib)


def test_substring_patterns_are_found():
    """Config-1-shaped draw (smaller text): every pattern cut from the text
    has count >= 1, and the counts sum to the number of matches."""
    w = workloads.config1(n=1 << 16)
    matches, counts = oracle.scan(w.patterns, w.text)
    t = w.text.tobytes()
    for j, p in enumerate(w.patterns):
        if t.find(p) >= 0:
            assert counts[j] >= 1
        else:
            assert counts[j] == 0
    assert int(counts.sum()) == matches.shape[0]


MUTANTS = {
    1: "output of a state not merged with the output of its failure state",
    2: "end position off by one",
    3: "every failure transition goes to the root",
    4: "character dropped on a failure instead of considered again",
    5: "failure function looks only one level up",
    6: "result ordered by id before position",
}


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistakes_are_caught(mutant, tmp_path):
    path = oracle.build_oracle(str(tmp_path / f"liboracle_m{mutant}.so"), mutant=mutant)
    lib = oracle.load(path)
    failures = []
    for chk in ALL_CHECKS:
        kw = {"cases": 400} if chk is check_random else {}
        failures += chk(lib, **kw)
    assert failures, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"
