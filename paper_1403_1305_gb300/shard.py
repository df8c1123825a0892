"""Splitting one scan across ranks (one GPU per rank) and merging the results.

Two splits, the paper's two architectures (Section III):

* ``text``: rank r owns end positions [lo_r, hi_r) of the text and scans
  text[max(0, lo_r - (m-1)) : hi_r] (m = longest pattern), keeping only
  matches that end in its range; the ranks' sorted lists concatenate in rank
  order and the counts add up.
* ``patterns``: rank r takes a contiguous id range of the patterns (its own
  machine) and scans the whole text; the sorted lists are merged by
  (position, id) and the counts, over disjoint ids, add up.

The scan of a rank's share is ``scanner(patterns, text) -> (matches,
counts)``; by default the library's ``ac_scan`` on the rank's GPU. The scan
path needs no exchange step, so the collectives here (gather of the matches,
sum of the counts over torch.distributed) run once, after the scans.
"""
from __future__ import annotations

import numpy as np


def text_ranges(n: int, world: int, warm: int):
    """Per rank: (scan start, first owned end position, end) for the text split."""
    out = []
    for r in range(world):
        lo, hi = r * n // world, (r + 1) * n // world
        out.append((max(0, lo - warm), lo, hi))
    return out


def pattern_ranges(P: int, world: int):
    """Per rank: contiguous pattern id range [lo, hi), sizes differing by at most 1."""
    return [(r * P // world, (r + 1) * P // world) for r in range(world)]


def merge_sorted(parts):
    """Merge (M_i, 2) uint32 arrays each sorted by (position, id)."""
    parts = [p for p in parts if p.shape[0]]
    if not parts:
        return np.zeros((0, 2), dtype=np.uint32)
    allm = np.concatenate(parts)
    order = np.lexsort((allm[:, 1], allm[:, 0]))
    return allm[order]


def _default_scanner(device: int):
    from . import ac as A

    def scan(patterns, text):
        a = A.ac_build(patterns, device=device)
        return A.ac_scan(a, text)

    return scan


def sharded_scan(patterns, text, split: str = "text", scanner=None, dist=None, device: int = 0):
    """Scan ``text`` for ``patterns`` split over the ranks of ``dist``
    (torch.distributed, initialised); every rank returns the full sorted
    matches and counts."""
    scanner = scanner or _default_scanner(device)
    world, rank = dist.get_world_size(), dist.get_rank()
    text = np.asarray(text, dtype=np.uint8)
    pats = [bytes(p) for p in patterns]
    P = len(pats)
    counts = np.zeros(P, dtype=np.int64)
    if split == "text":
        warm = max(len(p) for p in pats) - 1
        start, lo, hi = text_ranges(text.size, world, warm)[rank]
        m, c = scanner(pats, text[start:hi])
        m = m.copy()
        counts += np.asarray(c, dtype=np.int64)
        if m.shape[0]:
            m[:, 0] += start
            halo = m[:, 0] < lo        # owned by the previous rank
            np.subtract.at(counts, m[halo, 1].astype(np.int64), 1)
            m = m[~halo]
        parts = [None] * world
        dist.all_gather_object(parts, m)
        matches = np.concatenate([p for p in parts if p.shape[0]] or [np.zeros((0, 2), np.uint32)])
    elif split == "patterns":
        lo, hi = pattern_ranges(P, world)[rank]
        m = np.zeros((0, 2), np.uint32)
        if hi > lo:
            m, c = scanner(pats[lo:hi], text)
            m = m.copy()
            counts[lo:hi] = np.asarray(c, dtype=np.int64)
            if m.shape[0]:
                m[:, 1] += lo
        parts = [None] * world
        dist.all_gather_object(parts, m)
        matches = merge_sorted(parts)
    else:
        raise ValueError(f"unknown split {split!r}")
    import torch
    t = torch.from_numpy(counts)
    dist.all_reduce(t)
    return matches.astype(np.uint32), t.numpy().astype(np.uint64)
