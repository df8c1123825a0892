"""Seeded synthetic inputs for Aho-Corasick multi-pattern scanning.

This module only draws random texts and pattern sets (and packs DNA text into
2-bit codes as an input format); it holds none of the matching arithmetic.
It is the one piece of code that the oracle side and the CUDA side both use:
tests, ``bench.py`` and ``__graft_entry__.smoke()`` import it to create the
same inputs for both.

The shapes follow the workloads of the paper's setting (bio-computing texts:
DNA over {A,C,G,T}, protein over 20 amino-acid letters, Section I) and the
five benchmark configurations of this project:

  1. DNA 1 MiB, 100 patterns of length U[8,32] (50% cut from the text)
  2. DNA 256 MiB, 10,000 patterns of length U[16,64] (50% cut)
  3. protein 64 MiB, Zipf(0.5) letters, 100,000 patterns U[6,20] (70% cut)
  4. 4,096 DNA texts of log-uniform length [1 KiB, 4 MiB] against 8 pattern
     sets of 1,000..50,000 patterns U[12,40]
  5. a Poisson request stream over 16 pattern sets (8 DNA, 8 protein)

Every draw uses ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DNA = b"ACGT"
PROTEIN = b"ACDEFGHIKLMNPQRSTVWY"

MiB = 1 << 20


# --------------------------------------------------------------------------
# letters and texts
# --------------------------------------------------------------------------
def zipf_letters(rng: np.random.Generator, alphabet: bytes = PROTEIN, s: float = 0.5):
    """Letter order and probabilities for a Zipf(s) law over a seeded permutation.

    Rank k (1-based) gets probability proportional to k**-s; ranks are
    assigned to a random permutation of ``alphabet``.
    """
    letters = np.frombuffer(alphabet, dtype=np.uint8).copy()
    rng.shuffle(letters)
    w = np.arange(1, len(letters) + 1, dtype=np.float64) ** (-s)
    return letters, w / w.sum()


def iid_text(rng: np.random.Generator, n: int, letters: np.ndarray, probs=None) -> np.ndarray:
    """n i.i.d. letters (uint8 array); uniform when ``probs`` is None."""
    letters = np.asarray(letters, dtype=np.uint8)
    if probs is None:
        idx = rng.integers(0, len(letters), size=n, dtype=np.uint8)
    else:
        cdf = np.cumsum(probs)
        cdf[-1] = 1.0
        idx = np.searchsorted(cdf, rng.random(n), side="right").astype(np.uint8)
    return letters[idx]


def dna_text(rng: np.random.Generator, n: int) -> np.ndarray:
    return iid_text(rng, n, np.frombuffer(DNA, dtype=np.uint8))


def draw_patterns(rng, texts, P, lo, hi, frac_sub, letters, probs=None, exclude=None):
    """Draw exactly ``P`` distinct patterns with lengths uniform in [lo, hi].

    ``round(frac_sub * P)`` of them are substrings cut at uniform offsets of
    the given texts (a text is picked uniformly, weighted by nothing), the
    rest are i.i.d. letters. Duplicates are resampled. The two groups are
    shuffled together, so pattern ids mix both kinds.
    """
    if isinstance(texts, np.ndarray):
        texts = [texts]
    texts = [t for t in texts if len(t) >= lo]
    n_sub = int(round(frac_sub * P)) if texts else 0
    seen = set() if exclude is None else set(exclude)
    out = []
    letters = np.asarray(letters, dtype=np.uint8)
    tries = 0
    while len(out) < n_sub:
        tries += 1
        if tries > 100 * P + 1000:
            raise ValueError("cannot draw enough distinct substrings from these texts")
        t = texts[int(rng.integers(0, len(texts)))]
        L = int(rng.integers(lo, min(hi, len(t)) + 1))
        off = int(rng.integers(0, len(t) - L + 1))
        p = t[off:off + L].tobytes()
        if p not in seen:
            seen.add(p)
            out.append(p)
    while len(out) < P:
        tries += 1
        if tries > 200 * P + 2000:
            raise ValueError("cannot draw enough distinct patterns")
        L = int(rng.integers(lo, hi + 1))
        p = iid_text(rng, L, letters, probs).tobytes()
        if p not in seen:
            seen.add(p)
            out.append(p)
    order = rng.permutation(len(out))
    return [out[i] for i in order]


def random_patterns(rng, P, lo, hi, letters):
    """Exactly P distinct i.i.d. uniform patterns with lengths uniform in
    [lo, hi] (vectorised, for pattern sets of millions)."""
    letters = np.asarray(np.frombuffer(letters, np.uint8) if isinstance(letters, bytes) else letters, np.uint8)
    out, seen = [], set()
    while len(out) < P:
        k = P - len(out)
        lens = rng.integers(lo, hi + 1, size=k)
        mat = letters[rng.integers(0, len(letters), size=(k, hi), dtype=np.uint8)]
        for row, L in zip(mat, lens):
            b = row[:L].tobytes()
            if b not in seen:
                seen.add(b)
                out.append(b)
    return out


def embed(rng, text, patterns, count):
    """A copy of text with `count` patterns (drawn uniformly) written at
    uniform offsets."""
    t = np.array(text, dtype=np.uint8, copy=True)
    idx = rng.integers(0, len(patterns), size=count)
    for i in idx:
        p = np.frombuffer(patterns[int(i)], np.uint8)
        if p.size <= t.size:
            o = int(rng.integers(0, t.size - p.size + 1))
            t[o:o + p.size] = p
    return t


def pack2(text: np.ndarray, alphabet: bytes = DNA) -> np.ndarray:
    """Pack a text over a 4-letter alphabet into 2-bit codes, 4 per byte.

    Code k is the k-th letter of ``alphabet`` (A=0, C=1, G=2, T=3 for DNA);
    symbol i sits at bits 2*(i%4) of byte i//4 (least significant first).
    Bytes outside the alphabet are not representable and raise ValueError.
    """
    text = np.asarray(text, dtype=np.uint8)
    lut = np.full(256, 255, dtype=np.uint8)
    for k, b in enumerate(alphabet):
        lut[b] = k
    codes = lut[text]
    if codes.size and codes.max() == 255:
        raise ValueError("text holds a byte outside the 4-letter alphabet")
    pad = (-len(codes)) % 4
    if pad:
        codes = np.concatenate([codes, np.zeros(pad, np.uint8)])
    c = codes.reshape(-1, 4).astype(np.uint8)
    return (c[:, 0] | (c[:, 1] << 2) | (c[:, 2] << 4) | (c[:, 3] << 6)).astype(np.uint8)


def unpack2(packed: np.ndarray, n: int, alphabet: bytes = DNA) -> np.ndarray:
    """Inverse of :func:`pack2` for the first ``n`` symbols."""
    p = np.asarray(packed, dtype=np.uint8)
    c = np.stack([(p >> (2 * k)) & 3 for k in range(4)], axis=1).reshape(-1)[:n]
    return np.frombuffer(alphabet, dtype=np.uint8)[c]


# --------------------------------------------------------------------------
# benchmark configurations
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    text: np.ndarray
    patterns: list
    alphabet: bytes
    meta: dict = field(default_factory=dict)


def config1(seed: int = 1001, n: int = MiB, P: int = 100) -> Workload:
    """DNA 1 MiB, 100 patterns U[8,32], half cut from the text."""
    rng = np.random.default_rng(seed)
    text = dna_text(rng, n)
    pats = draw_patterns(rng, text, P, 8, 32, 0.5, np.frombuffer(DNA, np.uint8))
    return Workload("dna-1MiB-100pat", text, pats, DNA, {"seed": seed})


def config2(seed: int = 1002, n: int = 256 * MiB, P: int = 10_000) -> Workload:
    """DNA 256 MiB, 10,000 patterns U[16,64], half cut from the text."""
    rng = np.random.default_rng(seed)
    text = dna_text(rng, n)
    pats = draw_patterns(rng, text, P, 16, 64, 0.5, np.frombuffer(DNA, np.uint8))
    return Workload(f"dna-{n // MiB}MiB-{P}pat", text, pats, DNA, {"seed": seed})


def config3(seed: int = 1003, n: int = 64 * MiB, P: int = 100_000) -> Workload:
    """Protein 64 MiB (Zipf 0.5 letters), 100,000 patterns U[6,20], 70% cut."""
    rng = np.random.default_rng(seed)
    letters, probs = zipf_letters(rng)
    text = iid_text(rng, n, letters, probs)
    pats = draw_patterns(rng, text, P, 6, 20, 0.7, letters, probs)
    return Workload(f"protein-{n // MiB}MiB-{P}pat", text, pats, PROTEIN,
                    {"seed": seed, "letters": letters.tobytes(), "probs": probs})


def geometric_sizes(lo: int, hi: int, k: int):
    r = (hi / lo) ** (1.0 / (k - 1))
    return [int(round(lo * r ** i)) for i in range(k)]


def log_uniform_lengths(rng, count, lo, hi):
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


@dataclass
class BatchWorkload:
    name: str
    texts: list
    set_of_text: np.ndarray
    pattern_sets: list
    alphabet: bytes
    meta: dict = field(default_factory=dict)


def config4(seed: int = 1004, num_texts: int = 4096, lo: int = 1024, hi: int = 4 * MiB,
            num_sets: int = 8, set_lo: int = 1000, set_hi: int = 50_000,
            plen=(12, 40)) -> BatchWorkload:
    """4,096 DNA texts, log-uniform lengths, each paired with one of 8 pattern sets.

    Half of each set's patterns are cut from the texts paired with that set.
    """
    rng = np.random.default_rng(seed)
    lens = log_uniform_lengths(rng, num_texts, lo, hi)
    texts = [dna_text(rng, int(L)) for L in lens]
    set_of_text = rng.integers(0, num_sets, size=num_texts)
    sizes = geometric_sizes(set_lo, set_hi, num_sets) if num_sets > 1 else [set_lo]
    sets = []
    for k in range(num_sets):
        own = [texts[i] for i in np.flatnonzero(set_of_text == k)] or texts[:1]
        sets.append(draw_patterns(rng, own, sizes[k], plen[0], plen[1], 0.5,
                                  np.frombuffer(DNA, np.uint8)))
    return BatchWorkload(f"dna-batch-{num_texts}", texts, set_of_text, sets, DNA,
                         {"seed": seed, "total_bytes": int(lens.sum()), "set_sizes": sizes})


@dataclass
class ServeWorkload:
    name: str
    pattern_sets: list        # 16 lists of patterns
    set_alphabet: list        # alphabet bytes per set
    set_letters: list         # (letters, probs) per set for text draws
    meta: dict = field(default_factory=dict)


def config5_sets(seed: int = 1005, dna_sets=8, dna_P=5000, prot_sets=8, prot_P=20_000,
                 seed_text_len: int = 4 * MiB) -> ServeWorkload:
    """16 device-resident pattern sets: 8 DNA (5,000 x U[12,40]), 8 protein (20,000 x U[6,20]).

    Half of each set is cut from a seeded text of the set's kind so that the
    request texts (drawn the same way) hold matches.
    """
    rng = np.random.default_rng(seed)
    sets, alph, lets = [], [], []
    dna_l = np.frombuffer(DNA, np.uint8)
    for _ in range(dna_sets):
        src = dna_text(rng, seed_text_len)
        sets.append(draw_patterns(rng, src, dna_P, 12, 40, 0.5, dna_l))
        alph.append(DNA)
        lets.append((dna_l, None))
    for _ in range(prot_sets):
        letters, probs = zipf_letters(rng)
        src = iid_text(rng, seed_text_len, letters, probs)
        sets.append(draw_patterns(rng, src, prot_P, 6, 20, 0.5, letters, probs))
        alph.append(PROTEIN)
        lets.append((letters, probs))
    return ServeWorkload("serve-16sets", sets, alph, lets, {"seed": seed})


def request_stream(rng, rate_hz: float, count: int, num_sets: int = 16,
                   lo: int = 4096, hi: int = 64 * MiB):
    """Poisson arrivals: (arrival time s, set id, text length) for ``count`` requests."""
    gaps = rng.exponential(1.0 / rate_hz, size=count)
    t = np.cumsum(gaps)
    sets = rng.integers(0, num_sets, size=count)
    lens = log_uniform_lengths(rng, count, lo, hi)
    return t, sets, lens


# --------------------------------------------------------------------------
# tiny adversarial cases (for brute-force comparisons)
# --------------------------------------------------------------------------
def tiny_case(rng: np.random.Generator, alphabet: bytes = b"ab", max_n: int = 64,
              max_p: int = 8, max_len: int = 6, other_frac: float = 0.0):
    """A small random case: text over ``alphabet`` (plus optional out-of-alphabet
    bytes), patterns built to include prefixes, suffixes and duplicates of one
    another, and sometimes a pattern longer than the text.
    """
    letters = np.frombuffer(alphabet, dtype=np.uint8)
    n = int(rng.integers(0, max_n + 1))
    text = letters[rng.integers(0, len(letters), size=n)] if n else np.zeros(0, np.uint8)
    if n and other_frac > 0:
        mask = rng.random(n) < other_frac
        text = text.copy()
        text[mask] = ord("N") if alphabet != b"N" else ord("x")
    P = int(rng.integers(1, max_p + 1))
    pats = []
    for _ in range(P):
        kind = rng.integers(0, 5)
        if kind == 0 and pats:                       # duplicate
            pats.append(pats[int(rng.integers(0, len(pats)))])
        elif kind == 1 and pats:                     # prefix or suffix of another
            q = pats[int(rng.integers(0, len(pats)))]
            k = int(rng.integers(1, len(q) + 1))
            pats.append(q[:k] if rng.integers(0, 2) else q[-k:])
        elif kind == 2 and n:                        # cut from the text
            L = int(rng.integers(1, min(max_len, n) + 1))
            o = int(rng.integers(0, n - L + 1))
            cut = text[o:o + L]
            if (cut == ord("N")).any() or (cut == ord("x")).any():
                cut = letters[rng.integers(0, len(letters), size=L)]
            pats.append(cut.tobytes())
        elif kind == 3:                              # longer than the text
            L = n + int(rng.integers(1, 3))
            pats.append(letters[rng.integers(0, len(letters), size=L)].tobytes())
        else:
            L = int(rng.integers(1, max_len + 1))
            pats.append(letters[rng.integers(0, len(letters), size=L)].tobytes())
    return text, pats
