// Host construction of the matching machines (run once per pattern set).
//
// Steps, per pattern subset (Section II.A, Fig. 1; the folded table is the
// "AC-opt" machine of Section III / reference [4]):
//   1. goto function: insert the subset's patterns in their order, numbering
//      new states consecutively from root 0;
//   2. failure function breadth-first, folding each missing transition into
//      the transition of the failure state (so the table holds the complete
//      next-state function), and merging each state's output with the output
//      of its failure state;
//   3. states renumbered in breadth-first order so the shallow states, where
//      a walk over random text spends most of its time, form a prefix of the
//      table that the scan keeps in shared memory.
// Subsets (Section III's pattern-focused split, the paper's Fig. 5) are
// contiguous id ranges of as-equal-as-possible size, built on host threads.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>

#include "ac_internal.h"

namespace acgb {

namespace {

constexpr uint32_t kNone = 0xffffffffu;

// Failure-less machine (Section II.B; the paper's Section IV method): the
// goto function only, states renumbered breadth-first, each final state with
// its own patterns; missing transitions stay missing (kMissing).
int build_subset_pfac(const uint8_t *const *pats, const uint32_t *lens, uint32_t lo, uint32_t hi,
                      const uint8_t *sym, uint32_t sigma, HostSubset &S, std::string &why) {
    S.id_lo = lo;
    S.id_hi = hi;
    uint64_t chars = 0;
    for (uint32_t j = lo; j < hi; ++j) chars += lens[j];
    std::vector<uint32_t> child(sigma, kNone);
    child.reserve((chars + 1) * sigma);
    std::vector<uint32_t> depth(1, 0);
    depth.reserve(chars + 1);
    std::vector<std::pair<uint32_t, uint32_t>> finals;
    finals.reserve(hi - lo);
    uint64_t ns = 1;
    for (uint32_t j = lo; j < hi; ++j) {
        uint32_t s = 0;
        S.max_len = std::max(S.max_len, lens[j]);
        for (uint32_t k = 0; k < lens[j]; ++k) {
            const uint64_t idx = (uint64_t)s * sigma + sym[pats[j][k]];
            uint32_t t = child[idx];
            if (t == kNone) {
                if (ns >= (uint64_t)kMissing) {
                    why = "more than 2^31-2 states in one subset";
                    return AC_ERANGE;
                }
                t = (uint32_t)ns++;
                child[idx] = t;
                child.resize(ns * sigma, kNone);
                depth.push_back(depth[s] + 1);
            }
            s = t;
        }
        finals.emplace_back(s, j);
    }
    const uint32_t N = (uint32_t)ns;
    // breadth-first order over the goto edges
    std::vector<uint32_t> order;
    order.reserve(N);
    order.push_back(0);
    for (size_t h = 0; h < order.size(); ++h) {
        const uint64_t rr = (uint64_t)order[h] * sigma;
        for (uint32_t c = 0; c < sigma; ++c)
            if (child[rr + c] != kNone) order.push_back(child[rr + c]);
    }
    std::vector<uint32_t> rank(N);
    for (uint32_t i = 0; i < N; ++i) rank[order[i]] = i;
    // own patterns per state (ids ascending: inserted in id order)
    std::vector<uint32_t> cnt(N + 1, 0);
    for (auto &f : finals) cnt[rank[f.first] + 1]++;
    S.out_off.assign(N + 1, 0);
    for (uint32_t i = 0; i < N; ++i) S.out_off[i + 1] = S.out_off[i] + cnt[i + 1];
    S.out_ids.assign(finals.size(), 0);
    std::vector<uint32_t> fill(S.out_off.begin(), S.out_off.end() - 1);
    for (auto &f : finals) S.out_ids[fill[rank[f.first]]++] = f.second;
    S.states = N;
    S.table.resize((size_t)N * sigma);
    S.fail.assign(N, 0);  // not built: the failure-less machine has none
    S.depth.resize(N);
    for (uint32_t i = 0; i < N; ++i) {
        const uint32_t s = order[i];
        S.depth[i] = depth[s];
        const uint64_t rr = (uint64_t)s * sigma;
        uint32_t *dst = &S.table[(size_t)i * sigma];
        for (uint32_t c = 0; c < sigma; ++c) {
            const uint32_t t = child[rr + c];
            if (t == kNone) {
                dst[c] = kMissing;
            } else {
                const uint32_t nx = rank[t];
                dst[c] = nx | ((S.out_off[nx + 1] > S.out_off[nx]) ? kFlag : 0u);
            }
        }
    }
    return AC_OK;
}

int build_subset(const uint8_t *const *pats, const uint32_t *lens, uint32_t lo, uint32_t hi,
                 const uint8_t *sym, uint32_t sigma, HostSubset &S, std::string &why) {
    S.id_lo = lo;
    S.id_hi = hi;
    // 1. goto function (trie) with consecutive state numbers
    uint64_t chars = 0;
    for (uint32_t j = lo; j < hi; ++j) chars += lens[j];
    std::vector<uint32_t> child(sigma, kNone);
    child.reserve((chars + 1) * sigma);
    std::vector<uint32_t> depth(1, 0);
    depth.reserve(chars + 1);
    std::vector<std::pair<uint32_t, uint32_t>> finals;  // (state, pattern id)
    finals.reserve(hi - lo);
    uint64_t ns = 1;
    for (uint32_t j = lo; j < hi; ++j) {
        uint32_t s = 0;
        S.max_len = std::max(S.max_len, lens[j]);
        for (uint32_t k = 0; k < lens[j]; ++k) {
            uint32_t c = sym[pats[j][k]];
            uint64_t idx = (uint64_t)s * sigma + c;
            uint32_t t = child[idx];
            if (t == kNone) {
                if (ns >= (uint64_t)kStateMask) {
                    why = "more than 2^31-1 states in one subset";
                    return AC_ERANGE;
                }
                t = (uint32_t)ns++;
                child[idx] = t;
                child.resize(ns * sigma, kNone);
                depth.push_back(depth[s] + 1);
            }
            s = t;
        }
        finals.emplace_back(s, j);
    }
    const uint32_t N = (uint32_t)ns;

    // 2. breadth-first failure function with the missing transitions folded in
    std::vector<uint32_t> order;
    order.reserve(N);
    std::vector<uint32_t> fail(N, 0);
    order.push_back(0);
    for (uint32_t c = 0; c < sigma; ++c) {
        uint32_t t = child[c];
        if (t == kNone) {
            child[c] = 0;  // the root loops on symbols that start no pattern
        } else {
            fail[t] = 0;
            order.push_back(t);
        }
    }
    for (size_t h = 1; h < order.size(); ++h) {
        uint32_t r = order[h];
        uint64_t fr = (uint64_t)fail[r] * sigma, rr = (uint64_t)r * sigma;
        for (uint32_t c = 0; c < sigma; ++c) {
            uint32_t t = child[rr + c];
            if (t == kNone) {
                child[rr + c] = child[fr + c];
            } else {
                fail[t] = child[fr + c];
                order.push_back(t);
            }
        }
    }

    // breadth-first rank of every state
    std::vector<uint32_t> rank(N);
    for (uint32_t i = 0; i < N; ++i) rank[order[i]] = i;

    // output function: own patterns merged with the output of the failure state
    std::stable_sort(finals.begin(), finals.end(),
                     [](const std::pair<uint32_t, uint32_t> &x, const std::pair<uint32_t, uint32_t> &y) {
                         return x.first < y.first;
                     });
    std::vector<uint32_t> own_off(N + 1, 0);
    for (auto &f : finals) own_off[f.first + 1]++;
    for (uint32_t i = 0; i < N; ++i) own_off[i + 1] += own_off[i];
    S.out_off.assign(N + 1, 0);
    S.out_ids.clear();
    S.out_ids.reserve(finals.size() * 2);
    for (uint32_t i = 0; i < N; ++i) {
        const uint32_t t = order[i];
        // own ids: finals[own_off[t] .. own_off[t+1]) (ascending); merged with
        // the output of the failure state, which comes earlier in this order
        const size_t ob = own_off[t], oe = own_off[t + 1];
        size_t fb = 0, fe = 0;
        if (i > 0) {
            const uint32_t fr = rank[fail[t]];
            fb = S.out_off[fr];
            fe = S.out_off[fr + 1];
        }
        const size_t start = S.out_ids.size();
        S.out_ids.resize(start + (oe - ob) + (fe - fb));
        size_t a = ob, b = fb, w = start;
        while (a < oe && b < fe) {
            const uint32_t x = finals[a].second, y = S.out_ids[b];
            if (x <= y) {
                S.out_ids[w++] = x;
                ++a;
            } else {
                S.out_ids[w++] = y;
                ++b;
            }
        }
        while (a < oe) S.out_ids[w++] = finals[a++].second;
        while (b < fe) {
            const uint32_t y = S.out_ids[b++];
            S.out_ids[w++] = y;
        }
        if (S.out_ids.size() > 0xffffffffull) {
            why = "output function larger than 2^32 entries";
            return AC_ERANGE;
        }
        S.out_off[i + 1] = (uint32_t)S.out_ids.size();
    }

    // 3. renumbered dense table, with the output flag on each entry
    S.states = N;
    S.table.resize((size_t)N * sigma);
    S.fail.resize(N);
    S.depth.resize(N);
    for (uint32_t i = 0; i < N; ++i) {
        uint32_t s = order[i];
        S.fail[i] = rank[fail[s]];
        S.depth[i] = depth[s];
        uint64_t rr = (uint64_t)s * sigma;
        uint32_t *dst = &S.table[(size_t)i * sigma];
        for (uint32_t c = 0; c < sigma; ++c) {
            uint32_t nx = rank[child[rr + c]];
            uint32_t flag = (S.out_off[nx + 1] > S.out_off[nx]) ? kFlag : 0u;
            dst[c] = nx | flag;
        }
    }
    return AC_OK;
}

// Two-symbol table of a 4-letter machine: the composition of two transitions
// of the folded table (a multi-symbol step of the AC-opt machine), so a scan
// does one dependent lookup per two symbols. Column c1 + 4*c2 (the first
// symbol in the low bits, as in packed text). Bit 31: the state after both
// symbols has an output; bit 30: the state after c1 has one (the scan
// recovers that state from the one-symbol table when it must emit).
void build_table2(HostSubset &S) {
    const uint32_t N = S.states;
    S.table2.resize((size_t)N * 16);
    for (uint32_t s = 0; s < N; ++s) {
        const uint32_t *row = &S.table[(size_t)s * 4];
        uint32_t *dst = &S.table2[(size_t)s * 16];
        for (uint32_t c1 = 0; c1 < 4; ++c1) {
            const uint32_t m = row[c1];
            const uint32_t f1 = (m & kFlag) ? kFlag1 : 0u;
            const uint32_t *mrow = &S.table[(size_t)(m & kStateMask) * 4];
            for (uint32_t c2 = 0; c2 < 4; ++c2) {
                const uint32_t e = mrow[c2];
                dst[c1 + 4 * c2] = (e & kStateMask) | (e & kFlag) | f1;
            }
        }
    }
}

// 16-bit prefix of a 4-letter machine: the longest breadth-first prefix of
// rows whose next states all fit 15 bits, stored as (next << 1) | output
// flag, so shared memory holds twice the rows of the 32-bit table.
void build_table16(HostSubset &S) {
    uint32_t rows = 0;
    for (; rows < S.states; ++rows) {
        const uint32_t *row = &S.table[(size_t)rows * 4];
        if ((row[0] & kStateMask) > 0x7fffu || (row[1] & kStateMask) > 0x7fffu || (row[2] & kStateMask) > 0x7fffu ||
            (row[3] & kStateMask) > 0x7fffu)
            break;
    }
    S.rows16 = rows;
    S.table16.resize((size_t)rows * 4);
    for (size_t i = 0; i < S.table16.size(); ++i) {
        const uint32_t e = S.table[i];
        S.table16[i] = (uint16_t)(((e & 0x7fffu) << 1) | ((e & kFlag) ? 1u : 0u));
    }
}

// Escape-coded 16-bit prefix of a 4-letter machine (the lean scan's shared-
// memory table): entry = next state when it is below kEsc16 and its output is
// empty, else kEsc16, which sends the lookup to the 32-bit table in global
// memory (whose entry carries the output flag). Every row can be held this
// way, so the prefix is as long as shared memory allows (at most kRowsE16).
void build_table_e16(HostSubset &S) {
    const uint32_t rows = std::min<uint32_t>(S.states, kRowsE16);
    S.rows_e16 = rows;
    S.table_e16.resize((size_t)rows * 4);
    for (size_t i = 0; i < S.table_e16.size(); ++i) {
        const uint32_t e = S.table[i];
        const uint32_t next = e & kStateMask;
        S.table_e16[i] = (uint16_t)((next < kEsc16 && !(e & kFlag)) ? next : kEsc16);
    }
}

// Visit estimate for the placement choice: the probability of each state's
// string under i.i.d. letters with probabilities prob[] (a goto child's is
// its parent's times its letter's), summed over the states at or beyond each
// power of two of the breadth-first order.
void build_tail_mass(HostSubset &S, uint32_t sigma, const std::vector<double> &prob) {
    const uint32_t N = S.states;
    std::vector<double> p(N, 0.0);
    p[0] = 1.0;
    for (uint32_t s = 0; s < N; ++s)
        for (uint32_t c = 0; c < sigma; ++c) {
            const uint32_t t = S.table[(size_t)s * sigma + c] & kStateMask;
            if (S.depth[t] == S.depth[s] + 1) p[t] = p[s] * prob[c];  // goto child
        }
    std::vector<double> suffix(N + 1, 0.0);
    for (uint32_t s = N; s-- > 0;) suffix[s] = suffix[s + 1] + p[s];
    for (int k = 0; k < 32; ++k) S.tail_mass[k] = (1ull << k) < N ? suffix[1ull << k] : 0.0;
}

}  // namespace

int build_machines(const uint8_t *const *pats, const uint32_t *lens, uint32_t P, const ac_build_opts *opts,
                   ac_automaton *a) {
    auto t0 = std::chrono::steady_clock::now();
    if (!pats || !lens || P == 0) return set_error(AC_EINVAL, "ac_build: no patterns");
    for (uint32_t j = 0; j < P; ++j)
        if (lens[j] == 0 || !pats[j]) return set_error(AC_EINVAL, "ac_build: pattern %u is empty", j);

    // symbol map (a1): byte -> symbol, sigma = outside the alphabet
    memset(a->sym_of_byte, 0, sizeof(a->sym_of_byte));
    memset(a->byte_of_sym, 0, sizeof(a->byte_of_sym));
    bool used[256] = {false};
    uint32_t sigma = 0;
    if (opts && opts->alphabet) {
        const unsigned char *al = (const unsigned char *)opts->alphabet;
        for (size_t i = 0; al[i]; ++i) {
            if (used[al[i]]) return set_error(AC_EINVAL, "ac_build: alphabet repeats byte 0x%02x", al[i]);
            used[al[i]] = true;
            a->byte_of_sym[sigma++] = al[i];
        }
        if (sigma == 0) return set_error(AC_EINVAL, "ac_build: empty alphabet");
    } else {
        for (uint32_t j = 0; j < P; ++j)
            for (uint32_t k = 0; k < lens[j]; ++k) used[pats[j][k]] = true;
        for (int b = 0; b < 256; ++b)
            if (used[b]) a->byte_of_sym[sigma++] = (uint8_t)b;
    }
    if (sigma >= 256) return set_error(AC_ERANGE, "ac_build: alphabets of 256 symbols are not supported");
    for (int b = 0; b < 256; ++b) a->sym_of_byte[b] = (uint8_t)sigma;
    for (uint32_t s = 0; s < sigma; ++s) a->sym_of_byte[a->byte_of_sym[s]] = (uint8_t)s;
    for (uint32_t j = 0; j < P; ++j)
        for (uint32_t k = 0; k < lens[j]; ++k)
            if (a->sym_of_byte[pats[j][k]] == sigma)
                return set_error(AC_EINVAL, "ac_build: pattern %u holds byte 0x%02x outside the alphabet", j,
                                 pats[j][k]);
    a->sigma = sigma;
    a->dna_acgt = sigma == 4 && a->byte_of_sym[0] == 'A' && a->byte_of_sym[1] == 'C' &&
                  a->byte_of_sym[2] == 'G' && a->byte_of_sym[3] == 'T';
    a->P = P;
    a->max_len = 0;
    for (uint32_t j = 0; j < P; ++j) a->max_len = std::max(a->max_len, lens[j]);

    // two-symbol tables: asked for, or automatic for 4-letter DFA machines
    const uint32_t stride = opts ? opts->stride : 0;
    if (stride > 2) return set_error(AC_EINVAL, "ac_build: stride %u (0, 1 or 2)", stride);
    if (stride == 2 && (sigma != 4 || a->machine != AC_MACHINE_DFA))
        return set_error(AC_EINVAL, "ac_build: the two-symbol table needs a 4-letter alphabet and the DFA machine");
    const bool want2 = a->machine == AC_MACHINE_DFA && sigma == 4 && stride != 1;

    // letter frequencies of the patterns (add-one smoothed), for the visit estimate
    std::vector<double> prob(sigma, 1.0);
    double total = sigma;
    for (uint32_t j = 0; j < P; ++j)
        for (uint32_t k = 0; k < lens[j]; ++k) prob[a->sym_of_byte[pats[j][k]]] += 1.0;
    for (uint32_t j = 0; j < P; ++j) total += lens[j];
    for (auto &x : prob) x /= total;

    // subsets (a5)
    uint32_t K = (opts && opts->num_subsets) ? opts->num_subsets : 1;
    if (K > P) return set_error(AC_EINVAL, "ac_build: %u subsets for %u patterns", K, P);
    a->K = K;
    a->subs.assign(K, HostSubset());
    std::vector<int> rc(K, AC_OK);
    std::vector<std::string> why(K);
    const uint32_t builder = opts ? opts->builder : AC_BUILDER_HOST;
    if (builder > AC_BUILDER_DEVICE) return set_error(AC_EINVAL, "ac_build: unknown builder %u", builder);
    if (builder == AC_BUILDER_DEVICE && (a->machine != AC_MACHINE_DFA || a->device < 0))
        return set_error(AC_EINVAL, "ac_build: the device builder needs the DFA machine and a device");
    if (builder == AC_BUILDER_DEVICE) {
        // on the GPU, one subset after another; then the same derived tables
        int prev = -1;
        cudaGetDevice(&prev);
        if (cudaSetDevice(a->device) != cudaSuccess) return set_error(AC_ECUDA, "ac_build: cannot use device %d", a->device);
        for (uint32_t k = 0; k < K; ++k) {
            const uint32_t lo = (uint32_t)((uint64_t)k * P / K), hi = (uint32_t)((uint64_t)(k + 1) * P / K);
            try {
                rc[k] = build_subset_device(pats, lens, lo, hi, a->sym_of_byte, sigma, a->subs[k], why[k]);
            } catch (const std::bad_alloc &) {
                rc[k] = AC_ENOMEM;
                why[k] = "host allocation failed";
            }
            if (rc[k] != AC_OK) break;
        }
        if (prev >= 0 && prev != a->device) cudaSetDevice(prev);
        for (uint32_t k = 0; k < K; ++k)
            if (rc[k] != AC_OK) return set_error(rc[k], "ac_build: subset %u on the device: %s", k, why[k].c_str());
    }
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    unsigned nthr = std::min<unsigned>(K, hw);
    std::atomic<uint32_t> next{0};
    auto worker = [&]() {
        for (;;) {
            uint32_t k = next.fetch_add(1);
            if (k >= K) break;
            uint32_t lo = (uint32_t)((uint64_t)k * P / K), hi = (uint32_t)((uint64_t)(k + 1) * P / K);
            try {
                // (the device builder has built the subsets already; the derived tables follow here)
                if (builder != AC_BUILDER_DEVICE)
                    rc[k] = a->machine == AC_MACHINE_PFAC
                                ? build_subset_pfac(pats, lens, lo, hi, a->sym_of_byte, sigma, a->subs[k], why[k])
                                : build_subset(pats, lens, lo, hi, a->sym_of_byte, sigma, a->subs[k], why[k]);
                if (rc[k] == AC_OK && a->machine == AC_MACHINE_DFA) build_tail_mass(a->subs[k], sigma, prob);
                if (rc[k] == AC_OK && a->machine == AC_MACHINE_DFA && sigma == 4) {
                    build_table16(a->subs[k]);
                    build_table_e16(a->subs[k]);
                }
                if (rc[k] == AC_OK && stride == 2 && a->subs[k].states < kMaxStates2) build_table2(a->subs[k]);
            } catch (const std::bad_alloc &) {
                rc[k] = AC_ENOMEM;
                why[k] = "host allocation failed";
            }
        }
    };
    if (nthr <= 1) {
        worker();
    } else {
        std::vector<std::thread> th;
        for (unsigned i = 0; i < nthr; ++i) th.emplace_back(worker);
        for (auto &t : th) t.join();
    }
    for (uint32_t k = 0; k < K; ++k)
        if (rc[k] != AC_OK) return set_error(rc[k], "ac_build: subset %u: %s", k, why[k].c_str());
    if (want2 && stride == 0) {
        // automatic: only where a scan could choose it, i.e. a two-symbol
        // prefix of about 2,048 rows (what shared memory holds) keeps nearly
        // every visit (the same estimate the scan's choice uses)
        double worst = 0;
        for (auto &S : a->subs) worst = std::max(worst, S.tail_mass[11]);
        if (worst <= 0.02)
            for (auto &S : a->subs)
                if (S.states < kMaxStates2) build_table2(S);
    }
    a->has_table2 = want2;
    for (auto &S : a->subs) a->has_table2 = a->has_table2 && !S.table2.empty();
    if (stride == 2 && !a->has_table2)
        return set_error(AC_ERANGE, "ac_build: two-symbol table needs fewer than 2^28 states per subset");
    if (!a->has_table2)
        for (auto &S : a->subs) std::vector<uint32_t>().swap(S.table2);
    a->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return AC_OK;
}

}  // namespace acgb
