"""Host-side tests of the library (no GPU): exports, machine construction and
argument checks.

The machines are built with ``device=-1`` (host only) and walked here in
numpy, one symbol at a time, and the walk is compared with the oracle; this
checks the trie, the breadth-first failure function, the output merge, the
fold into a dense table and the renumbering without any CUDA code running.
"""
import os
import re

import numpy as np
import pytest

import oracle
import workloads
from paper_1403_1305_gb300 import ac as A

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ac.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^AC_API\s+[\w\s\*]*?\b(ac_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_function():
    lib = A.lib()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(A.EXPORTED)


def test_version_and_strerror():
    assert A.ac_version() >= 10000
    assert A.ac_strerror(A.AC_ERANGE) == "size out of range"
    assert A.ac_strerror(12345) == "unknown error"


def walk(a, text):
    """Scan `text` with the library's host tables (all subsets), in numpy."""
    st = A.ac_stats(a)
    res = []
    for k in range(st["num_subsets"]):
        v = A.ac_subset(a, k)
        T, off, ids, sym = v["table"], v["out_off"], v["out_ids"], v["symbol_of_byte"]
        sigma = v["sigma"]
        s = 0
        tb = np.frombuffer(text, np.uint8) if isinstance(text, bytes) else np.asarray(text, dtype=np.uint8)
        for i, b in enumerate(tb.tolist()):
            c = sym[b]
            e = int(T[s, c]) if c < sigma else 0
            s = e & 0x7FFFFFFF
            if e >> 31:
                res += [(i, int(j)) for j in ids[off[s]:off[s + 1]]]
            else:
                assert off[s + 1] == off[s]
    res.sort()
    return np.asarray(res, dtype=np.uint32).reshape(-1, 2)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_host_tables_match_oracle_on_random_cases(K):
    rng = np.random.default_rng(100 + K)
    for i in range(300):
        text, pats = workloads.tiny_case(rng, b"ACGT" if i % 2 else b"ab", max_n=80, max_p=9, max_len=6,
                                         other_frac=0.1 if i % 4 == 0 else 0.0)
        if len(pats) < K:
            continue
        a = A.ac_build(pats, num_subsets=K, device=-1)
        want, _ = oracle.scan(pats, text)
        assert np.array_equal(walk(a, text), want), (i, pats, bytes(text))


def test_worked_examples_on_host_tables():
    for pats, text, want in (([b"AB", b"ABG", b"BEDE", b"EF"], b"ABEDE", [[1, 0], [4, 2]]),
                             ([b"HE", b"HIS", b"SHE", b"HERS"], b"USHERS", [[3, 0], [3, 2], [5, 3]])):
        a = A.ac_build(pats, device=-1)
        assert walk(a, text).tolist() == want


def test_breadth_first_numbering_and_failure_function():
    w = workloads.config1(n=1 << 14, P=60)
    a = A.ac_build(w.patterns, alphabet="ACGT", device=-1)
    v = A.ac_subset(a, 0)
    m = oracle.Machine(w.patterns)
    assert v["states"] == m.num_states           # same goto function, renumbered
    depth, fail = v["depth"], v["fail"]
    assert depth[0] == 0 and fail[0] == 0
    assert np.all(np.diff(depth.astype(np.int64)) >= 0)     # breadth-first order
    assert np.all(depth[fail[1:]] < depth[1:])             # failure goes shallower
    # every state's output holds exactly the patterns that are suffixes of its string
    strings = {0: b""}
    T = v["table"]
    for s in range(v["states"]):
        for c in range(4):
            t = int(T[s, c]) & 0x7FFFFFFF
            if depth[t] == depth[s] + 1 and t not in strings:
                strings[t] = strings[s] + b"ACGT"[c:c + 1]
    assert len(strings) == v["states"]
    off, ids = v["out_off"], v["out_ids"]
    for s, string in list(strings.items())[:400]:
        want = sorted(j for j, p in enumerate(w.patterns) if string.endswith(p))
        assert ids[off[s]:off[s + 1]].tolist() == want


def test_subset_split_is_contiguous_and_balanced():
    pats = [bytes([65 + i % 4]) * (1 + i // 4) for i in range(10)]
    a = A.ac_build(pats, num_subsets=4, device=-1)
    ranges = [(A.ac_subset(a, k)["id_lo"], A.ac_subset(a, k)["id_hi"]) for k in range(4)]
    assert ranges[0][0] == 0 and ranges[-1][1] == 10
    assert all(ranges[i][1] == ranges[i + 1][0] for i in range(3))
    sizes = [h - l for l, h in ranges]
    assert max(sizes) - min(sizes) <= 1


def test_argument_errors():
    with pytest.raises(A.AcError) as e:
        A.ac_build([], device=-1)
    assert e.value.code == A.AC_EINVAL
    with pytest.raises(A.AcError) as e:
        A.ac_build([b"A", b""], device=-1)
    assert e.value.code == A.AC_EINVAL
    with pytest.raises(A.AcError) as e:
        A.ac_build([b"A", b"C"], num_subsets=3, device=-1)
    assert e.value.code == A.AC_EINVAL
    with pytest.raises(A.AcError) as e:
        A.ac_build([b"ACGN"], alphabet="ACGT", device=-1)
    assert e.value.code == A.AC_EINVAL
    with pytest.raises(A.AcError) as e:
        A.ac_build([b"AC"], alphabet="AAC", device=-1)
    assert e.value.code == A.AC_EINVAL
    a = A.ac_build([b"AC"], device=-1)
    with pytest.raises(A.AcError) as e:
        A.ac_scan(a, b"ACAC")                 # host-only automaton cannot scan
    assert e.value.code == A.AC_EINVAL
    with pytest.raises(A.AcError):
        A.ac_set_scan_config(a, threads=48)
    with pytest.raises(A.AcError):
        A.ac_set_scan_config(a, chains=3)
    with pytest.raises(A.AcError):
        A.ac_set_scan_config(a, kernel=5)
    # the device builder needs a device and the folded machine; unknown builders are refused
    for kw in (dict(device=-1), dict(device=-1, machine=A.AC_MACHINE_PFAC)):
        with pytest.raises(A.AcError) as e:
            A.ac_build([b"AC"], builder=A.AC_BUILDER_DEVICE, **kw)
        assert e.value.code == A.AC_EINVAL
    with pytest.raises(A.AcError) as e:
        A.ac_build([b"AC"], builder=9, device=-1)
    assert e.value.code == A.AC_EINVAL
    # the launch probe refuses empty or oversized launches before touching a device
    for args in ((0, 1, 32), (1, 0, 32), (1, 1, 0), (1, 1, 1025)):
        with pytest.raises(A.AcError) as e:
            A.ac_probe_launch(None, *args)
        assert e.value.code == A.AC_EINVAL


def test_explicit_alphabet_order_sets_symbol_codes():
    a = A.ac_build([b"GATTACA"], alphabet="ACGT", device=-1)
    sym = A.ac_subset(a, 0)["symbol_of_byte"]
    assert [sym[ord(c)] for c in "ACGT"] == [0, 1, 2, 3]
    assert sym[ord("N")] == 4


def pfac_walk(a, text):
    """The failure-less walk of Section II.B from every start, on the library's host table."""
    v = A.ac_subset(a, 0)
    T, off, ids, sym, sg = v["table"], v["out_off"], v["out_ids"], v["symbol_of_byte"], v["sigma"]
    tb = np.frombuffer(text, np.uint8) if isinstance(text, bytes) else np.asarray(text, np.uint8)
    res = []
    for st in range(tb.size):
        s = 0
        for k in range(st, tb.size):
            c = sym[tb[k]]
            if c >= sg:
                break
            e = int(T[s, c])
            if e == 0x7FFFFFFF:
                break
            s = e & 0x7FFFFFFF
            if e >> 31:
                res += [(k, int(j)) for j in ids[off[s]:off[s + 1]]]
    res.sort()
    return np.asarray(res, np.uint32).reshape(-1, 2)


def test_failure_less_machine_tables():
    """AC_MACHINE_PFAC builds the goto function only; walking it from every
    start position gives the oracle's result, and Fig. 6's state numbers hold
    after breadth-first renumbering of the same trie."""
    rng = np.random.default_rng(31)
    for i in range(300):
        text, pats = workloads.tiny_case(rng, b"ACGT" if i % 2 else b"ab", max_n=60, max_p=8, max_len=6,
                                         other_frac=0.05)
        a = A.ac_build(pats, device=-1, machine=A.AC_MACHINE_PFAC)
        assert np.array_equal(pfac_walk(a, text), oracle.scan(pats, text)[0]), (i, pats)
    a = A.ac_build([b"HE", b"HIS", b"SHE", b"HERS"], device=-1, machine=A.AC_MACHINE_PFAC)
    assert pfac_walk(a, b"USHERS").tolist() == [[3, 0], [3, 2], [5, 3]]
    assert A.ac_stats(a)["states"] == oracle.Machine([b"HE", b"HIS", b"SHE", b"HERS"], False).num_states


def walk2(a, text):
    """Scan `text` two symbols per lookup with the library's two-symbol host
    tables (pairs holding a byte outside the alphabet, and a ragged last
    symbol, go through the one-symbol table), in numpy."""
    res = []
    for k in range(A.ac_stats(a)["num_subsets"]):
        v = A.ac_subset(a, k)
        T, T2, off, ids, sym = v["table"], v["table2"], v["out_off"], v["out_ids"], v["symbol_of_byte"]
        tb = np.frombuffer(text, np.uint8).tolist() if isinstance(text, bytes) else list(text)
        s = 0

        def step(s, i):
            c = sym[tb[i]]
            e = int(T[s, c]) if c < 4 else 0
            if e >> 31:
                res.extend((i, int(j)) for j in ids[off[e & 0x7FFFFFFF]:off[(e & 0x7FFFFFFF) + 1]])
            return e & 0x7FFFFFFF

        i = 0
        while i < len(tb):
            c1 = sym[tb[i]]
            c2 = sym[tb[i + 1]] if i + 1 < len(tb) else 4
            if c1 < 4 and c2 < 4:
                e = int(T2[s, c1 + 4 * c2])
                mid = int(T[s, c1]) & 0x7FFFFFFF
                assert bool(e & (1 << 30)) == (off[mid + 1] > off[mid])
                if e & (1 << 30):
                    res.extend((i, int(j)) for j in ids[off[mid]:off[mid + 1]])
                s = e & 0x3FFFFFFF
                assert bool(e >> 31) == (off[s + 1] > off[s])
                if e >> 31:
                    res.extend((i + 1, int(j)) for j in ids[off[s]:off[s + 1]])
                i += 2
            else:
                s = step(s, i)
                i += 1
    res.sort()
    return np.asarray(res, dtype=np.uint32).reshape(-1, 2)


def test_two_symbol_tables_match_oracle():
    """The two-symbol table (built automatically for 4-letter alphabets):
    a pair-wise walk over it gives the oracle's matches, including texts of
    odd length and bytes outside the alphabet."""
    rng = np.random.default_rng(77)
    checked = 0
    for i in range(300):
        text, pats = workloads.tiny_case(rng, b"ACGT", max_n=81, max_p=9, max_len=7,
                                         other_frac=0.1 if i % 3 == 0 else 0.0)
        K = 1 + i % 2 if len(pats) >= 2 else 1
        a = A.ac_build(pats, alphabet="ACGT", num_subsets=K, device=-1)
        assert A.ac_subset(a, 0)["table2"] is not None
        assert A.ac_stats(a)["table2_bytes"] == 4 * A.ac_stats(a)["table_bytes"]
        assert np.array_equal(walk2(a, text), oracle.scan(pats, text)[0]), (i, pats, bytes(text))
        checked += 1
    assert checked == 300


def test_two_symbol_table_options():
    pats = [b"ACG", b"GT", b"TTA"]
    assert A.ac_subset(A.ac_build(pats, alphabet="ACGT", device=-1, stride=1), 0)["table2"] is None
    assert A.ac_stats(A.ac_build(pats, alphabet="ACGT", device=-1, stride=1))["table2_bytes"] == 0
    assert A.ac_subset(A.ac_build(pats, alphabet="ACGT", device=-1, stride=2), 0)["table2"] is not None
    assert A.ac_subset(A.ac_build([b"ab", b"ba"], device=-1), 0)["table2"] is None       # 2 letters
    assert A.ac_subset(A.ac_build(pats, alphabet="ACGT", device=-1, machine=A.AC_MACHINE_PFAC), 0)["table2"] is None
    for kw in (dict(alphabet="ACGTN", stride=2), dict(alphabet="ACGT", stride=3),
               dict(alphabet="ACGT", stride=2, machine=A.AC_MACHINE_PFAC)):
        with pytest.raises(A.AcError) as e:
            A.ac_build(pats, device=-1, **kw)
        assert e.value.code == A.AC_EINVAL
    a = A.ac_build(pats, alphabet="ACGT", device=-1, stride=1)
    with pytest.raises(A.AcError):
        A.ac_set_scan_config(a, stride=2)
    with pytest.raises(A.AcError):
        A.ac_set_scan_config(a, stride=5)
    A.ac_set_scan_config(a, stride=1)


def test_sixteen_bit_prefix():
    """The 16-bit prefix holds (next << 1) | output bit for the longest
    breadth-first prefix of rows whose next states fit 15 bits."""
    w = workloads.config2(n=1 << 20, P=3000)
    a = A.ac_build(w.patterns, alphabet="ACGT", device=-1)
    v = A.ac_subset(a, 0)
    T, T16 = v["table"], v["table16"]
    r = T16.shape[0]
    assert 0 < r < v["states"]
    assert np.array_equal(T16.astype(np.uint32) >> 1, T[:r] & 0x7FFFFFFF)
    assert np.array_equal(T16.astype(np.uint32) & 1, T[:r] >> 31)
    assert (T[r] & 0x7FFFFFFF).max() > 0x7FFF      # the next row does not fit
    assert A.ac_subset(A.ac_build([b"ab", b"ba"], device=-1), 0)["table16"] is None
    small = A.ac_subset(A.ac_build([b"ACGT", b"GA"], alphabet="ACGT", device=-1), 0)
    assert small["table16"].shape[0] == small["states"]


def walk_e16(v, text, hot):
    """Scan with the escape-coded 16-bit prefix as the lean kernel reads it:
    a state below `hot` reads its 16-bit entry, an escape (or a state at or
    beyond `hot`) reads the 32-bit table, whose entry carries the output bit."""
    T, E, off, ids, sym = v["table"], v["table_e16"], v["out_off"], v["out_ids"], v["symbol_of_byte"]
    res, s = [], 0
    for i, b in enumerate(np.asarray(text, dtype=np.uint8).tolist()):
        c = int(sym[b])
        if c >= 4:
            s = 0
            continue
        e = int(E[s, c]) if s < hot else 0xFFFF
        if e == 0xFFFF:
            e = int(T[s, c])
        s = e & 0x7FFFFFFF
        if e >> 31:
            res += [(i, int(j)) for j in ids[off[s]:off[s + 1]]]
    res.sort()
    return np.asarray(res, dtype=np.uint32).reshape(-1, 2)


def test_escape_coded_prefix():
    """The lean kernel's shared-memory table: rows [0, min(states, 32768)),
    entry = next state when it is below 65,535 and has an empty output, else
    the escape 65,535. A machine wide enough that prefix rows lead to states
    beyond 65,535 (100,000 patterns) has both kinds of escape; walking it with
    prefixes of several lengths gives the oracle's matches."""
    rng = np.random.default_rng(1600)
    text = workloads.dna_text(rng, 60_000)
    pats = workloads.draw_patterns(rng, text, 100_000, 12, 20, 0.5, np.frombuffer(b"ACGT", np.uint8))
    pats += [b"ACG", b"TTAG", b"GATTA"]   # outputs at shallow states
    a = A.ac_build(pats, alphabet="ACGT", device=-1)
    v = A.ac_subset(a, 0)
    T, E = v["table"], v["table_e16"]
    r = E.shape[0]
    assert r == min(v["states"], 1 << 15) and v["states"] > 1 << 16
    nxt, flag = T[:r] & 0x7FFFFFFF, T[:r] >> 31
    want_e = np.where((nxt < 0xFFFF) & (flag == 0), nxt, 0xFFFF)
    assert np.array_equal(E.astype(np.uint32), want_e)
    assert ((nxt >= 0xFFFF) & (E == 0xFFFF)).any() and ((flag == 1) & (E == 0xFFFF)).any()
    want = oracle.scan(pats, text)[0]
    for hot in (0, 5, 1000, r):
        assert np.array_equal(walk_e16(v, text[:20_000] if hot < r else text, hot),
                              oracle.scan(pats, text[:20_000] if hot < r else text)[0])
    assert want.shape[0] > 0
    assert A.ac_subset(A.ac_build([b"ab", b"ba"], device=-1), 0)["table_e16"] is None


def test_results_take_moves_results_into_flat_arrays():
    """ac_results_take (host only): the matches and counts of several results
    land in two flat arrays at the offsets it reports, and the results are
    released (zeroed)."""
    import ctypes as C
    libc = C.CDLL(None)
    libc.malloc.restype = C.c_void_p
    libc.malloc.argtypes = [C.c_size_t]
    rng = np.random.default_rng(5)
    shapes = [(3, 4, True), (0, 2, False), (5, 0, False), (0, 0, False), (7, 3, True)]
    outs = (A.ac_result * len(shapes))()
    want_m, want_c = [], []
    for i, (m, P, with_counts) in enumerate(shapes):
        mm = rng.integers(0, 1 << 31, size=(m, 2)).astype(np.uint32)
        cc = rng.integers(0, 1000, size=P).astype(np.uint64) if with_counts else np.zeros(P, np.uint64)
        want_m.append(mm)
        want_c.append(cc)
        if m:
            p = libc.malloc(8 * m)
            C.memmove(p, mm.ctypes.data, 8 * m)
            outs[i].matches = C.cast(p, C.POINTER(A.ac_match))
        outs[i].num_matches = m
        if with_counts:
            q = libc.malloc(8 * P)
            C.memmove(q, cc.ctypes.data, 8 * P)
            outs[i].counts = C.cast(q, C.POINTER(C.c_uint64))
        outs[i].num_patterns = P
    got = A._take_results(outs, len(shapes), True)
    for (gm, gc), wm, wc in zip(got, want_m, want_c):
        assert np.array_equal(gm, wm) and gm.shape == wm.shape
        assert np.array_equal(gc, wc)
    for i in range(len(shapes)):
        assert outs[i].num_matches == 0 and not outs[i].matches and not outs[i].counts
    # without counts; and the NULL-argument refusal
    outs2 = (A.ac_result * 1)()
    outs2[0].num_patterns = 9
    [(m, c)] = A._take_results(outs2, 1, False)
    assert m.shape == (0, 2) and c is None
    assert A.lib().ac_results_take(None, 1, None, None, None, None) == A.AC_EINVAL


def test_ac_log_levels():
    """AC_LOG=2 prints the build line and errors on stderr, AC_LOG=1 errors
    only, unset nothing (host-only automata: no GPU needed)."""
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1403_1305_gb300 import ac as A\n"
            "A.ac_build([b'AC', b'GT'], alphabet='ACGT', device=-1)\n"
            "try:\n"
            "    A.ac_build([b'AX'], alphabet='ACGT', device=-1)\n"
            "except A.AcError:\n"
            "    pass\n") % os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    def run(level):
        env = dict(os.environ)
        env.pop("AC_LOG", None)
        if level is not None:
            env["AC_LOG"] = str(level)
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        return [l for l in r.stderr.splitlines() if l.startswith("acgb300:")]
    two = run(2)
    assert any("build: 2 patterns" in l for l in two)
    assert any("error -1" in l and "outside the alphabet" in l for l in two)
    one = run(1)
    assert one and all("error" in l for l in one)
    assert run(None) == []


def _views(a):
    st = A.ac_stats(a)
    out = []
    for k in range(st["num_subsets"]):
        v = A.ac_subset(a, k)
        out.append({f: (None if v[f] is None else np.asarray(v[f]).copy()) if isinstance(v[f], np.ndarray) or v[f] is None
                     else v[f] for f in v})
    return st, out


def _same_machines(a, b):
    sa, va = _views(a)
    sb, vb = _views(b)
    for f in ("num_patterns", "num_subsets", "sigma", "max_len", "states", "table_bytes", "output_entries",
              "table2_bytes"):
        assert sa[f] == sb[f], f
    for x, y in zip(va, vb):
        assert x.keys() == y.keys()
        for f in x:
            if isinstance(x[f], np.ndarray):
                assert isinstance(y[f], np.ndarray) and np.array_equal(x[f], y[f]), f
            else:
                assert x[f] == y[f], f


def test_save_and_load_round_trip(tmp_path):
    """ac_save / ac_load (host-only automata: no GPU needed): the loaded
    machines equal the saved ones table for table, for one machine, subsets,
    the two-symbol table, the failure-less machine and a 20-letter alphabet."""
    rng = np.random.default_rng(12)
    text, pats = workloads.tiny_case(rng, b"ACGT", max_n=3000, max_p=40, max_len=12)
    prot = [bytes(rng.choice(np.frombuffer(workloads.PROTEIN, np.uint8), size=int(rng.integers(2, 9))))
            for _ in range(50)]
    cases = [dict(patterns=pats, alphabet="ACGT"), dict(patterns=pats, alphabet="ACGT", num_subsets=3),
             dict(patterns=pats, alphabet="ACGT", stride=2), dict(patterns=pats, alphabet="ACGT",
                                                                 machine=A.AC_MACHINE_PFAC),
             dict(patterns=prot, alphabet=workloads.PROTEIN)]
    for i, kw in enumerate(cases):
        a = A.ac_build(device=-1, **kw)
        path = tmp_path / f"m{i}.acm"
        A.ac_save(a, path)
        b = A.ac_load(path, device=-1)
        _same_machines(a, b)


def test_load_refuses_bad_files(tmp_path):
    pats = [b"ACGT", b"CG", b"TTA"]
    a = A.ac_build(pats, alphabet="ACGT", device=-1)
    good = tmp_path / "good.acm"
    A.ac_save(a, good)
    data = good.read_bytes()

    def refused(blob, name):
        p = tmp_path / name
        p.write_bytes(blob)
        with pytest.raises(A.AcError) as e:
            A.ac_load(p, device=-1)
        assert e.value.code == A.AC_EINVAL

    refused(data[:-5], "truncated.acm")
    refused(data + b"\0", "trailing.acm")
    refused(b"NOTAFILE" + data[8:], "magic.acm")
    # the first table entry (after the header and the subset's scalars) points past the machine
    first = 8 + 4 + 16 + 8 + 4 + 2 + 512 + 8 + 24 + 32 * 8 + 8
    bad = bytearray(data)
    bad[first:first + 4] = (0x7FFFFFF0).to_bytes(4, "little")
    refused(bytes(bad), "transition.acm")
    # header: magic 8, format 4, P K sigma max_len placement machine smem_cap (4 each), ACGT flag, table2
    # flag, then sym_of_byte[256] and byte_of_sym[256]
    flag, sym, inv = 8 + 4 + 7 * 4, 8 + 4 + 7 * 4 + 2, 8 + 4 + 7 * 4 + 2 + 256
    assert data[flag] == 1 and data[inv:inv + 4] == b"ACGT" and data[sym + ord("A")] == 0
    bad = bytearray(data)
    bad[flag] = 0                                   # ACGT flag that disagrees with the alphabet
    refused(bytes(bad), "acgt_flag.acm")
    bad = bytearray(data)
    bad[sym + ord("A")], bad[sym + ord("C")] = 1, 0  # map no longer inverted by byte_of_sym
    refused(bytes(bad), "inverse.acm")
    bad = bytearray(data)
    bad[sym + ord("N")] = 2                          # a second byte for symbol 2
    refused(bytes(bad), "two_bytes.acm")
    with pytest.raises(A.AcError) as e:
        A.ac_load(tmp_path / "missing.acm", device=-1)
    assert e.value.code == A.AC_EINVAL
