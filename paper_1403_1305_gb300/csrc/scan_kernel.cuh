// The scan: one dependent goto-table lookup per text symbol per machine.
//
// What is computed (Section II.A of the paper, with the failure transitions
// folded into the table as in the AC-opt machine of Section III): from state
// s, symbol c leads to table[s][c]; an entry with bit 31 set leads to a state
// whose output is not empty, and every pattern of that output ends at the
// current position.
//
// Parallel decomposition (Section III, both architectures of reference [2]):
//  * input-focused: the text is cut into rows of `row_bytes` bytes. A chain
//    (one thread's walk) owns the end positions of one row and starts from
//    the root `warm` symbols (longest pattern - 1) before the row, rounded up
//    to whole stages; a walk that starts that early reaches, at every owned
//    position, the same state as a walk from the text start would as far as
//    the output is concerned (every pattern ending there starts inside the
//    warm-up), so no match is lost or duplicated.
//  * pattern-focused: subset machine k of K scans the same text; tiles are
//    (row block, subset) pairs with the subset index varying fastest so
//    concurrent CTAs share text rows in L2.
//
// GB300 mapping:
//  * persistent CTAs (one per SM by default) loop over tiles;
//  * the breadth-first prefix of the subset's table (the shallow states the
//    walk visits most) is copied into shared memory once per tile change;
//    deeper states are read through L2 (hybrid placement);
//  * each warp runs its own text pipeline: every lane issues a 1-D bulk async
//    copy (cp.async.bulk, the TMA engine) of the next 32 bytes of each of its
//    C chains into a per-warp shared-memory slot, completing on an mbarrier
//    with a transaction count; NS slots are in flight;
//  * lanes walk 16 symbols per sub-block from registers, OR-ing the entries;
//    only a sub-block whose OR shows an output flag (or a text edge, or a
//    byte outside the alphabet) is walked again symbol by symbol, with all 32
//    lanes together, and its matches are appended through one atomicAdd per
//    warp (ballot + warp prefix sum of the output sizes);
//  * every mbarrier wait is bounded (2 s of global time); on expiry the
//    kernel records an error word and stops issuing work.
#pragma once

#include <cuda.h>

#include "ac_internal.h"

namespace acgb {
namespace kern {

constexpr int kNS = 2;           // pipeline slots per warp
constexpr uint32_t kSB = 16;     // bytes per sub-block
constexpr unsigned kFull = 0xffffffffu;

enum { FMT_U8 = 0, FMT_P2 = 1 };
enum { ALPHA_MAP = 0, ALPHA_ACGT = 1 };
// table placement of a launch: all rows in shared memory; a breadth-first
// prefix in shared memory and the rest read through L2; a power-of-two
// prefix read optimistically (see lookup); or, for 4-letter machines, a
// prefix of 16-bit entries (ld_hybrid16) and the rest read through L2
enum { MODE_SMEM = 0, MODE_HYBRID = 1, MODE_OPT = 2, MODE_H16 = 3 };

// What a chain needs to know about the text its row belongs to.
struct ChainText {
    uint64_t row_in_text;  // row index within its text
    uint64_t nsym;         // symbols of its text
    uint64_t vbase;        // key position of the text's first symbol
    uint64_t cbase;        // counts offset of the text
};

struct ScanParams {
    const uint8_t *text;
    uint64_t nbytes;        // bytes of text
    uint64_t nsym;          // symbols
    uint64_t full_rows;     // rows of row_bytes entirely inside the text (2-D tensor map)
    uint64_t num_rows;      // full_rows, plus one if a partial last row exists
    uint64_t row_begin;     // rows [row_begin, row_end) are this launch's (single text; a batch: all rows)
    uint64_t row_end;
    uint64_t num_tiles;
    uint32_t row_bytes;     // multiple of kStageBytes
    uint32_t rows_per_tile; // warps * 32 * C
    uint32_t K;
    uint32_t sigma;
    uint32_t smem_rows;     // table rows that fit in shared memory
    uint32_t table_words;   // words reserved for the table in shared memory
    uint32_t key_shift;     // key = pos << key_shift | id
    uint32_t tail_bytes;    // bytes of the partial last row (1-D tensor map), 0 if none
    const SubsetDev *subs;
    unsigned long long *keys;
    uint64_t cap;
    unsigned long long *num;
    unsigned long long *counts;
    uint32_t *err;
    uint64_t wait_ns;       // limit of every bounded device-side wait; 0 gives up at the first wait
    EmitEntry *q;           // lean kernel: scratch for the queue of stages to emit, split between warps
    uint64_t q_cap;         // (null: stages with matches are walked again in place)
    // batch mode (several texts in one arena of whole rows)
    const BatchItemDev *items;  // sorted by first row
    const BatchTileDev *tiles;  // one per tile: machine and first row
    uint32_t num_items;
    uint8_t sym_of_byte[256];
    // short-text kernel: the machine's descriptor (a copy of subs[0])
    SubsetDev sub0;
};

// ------------------------------------------------------------------ PTX helpers
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start before the launch ahead of it in the stream has
// finished; pdl_wait() returns once that launch has completed and its writes
// are visible (at once for a kernel launched without the attribute), and
// pdl_release() lets the launch behind this one start early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" :::); }

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// L2 eviction policies: the text streams through once (evict first), the
// goto table is re-read all the time (evict last), so the text does not push
// the table out of L2.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y, uint64_t *bar,
                                            uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void tma_load_1d(void *dst, const CUtensorMap *map, int32_t x, uint64_t *bar,
                                            uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2}], [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

// table entry read through L2 with the evict-last policy
__device__ __forceinline__ uint32_t ld_table(const uint32_t *p, uint64_t pol) {
    uint32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: false (and the error word set) once
// `limit` ns have passed; a limit of 0 gives up before the first check.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, uint32_t *err, uint64_t limit) {
    if (limit == 0) {
        atomicOr(err, 1u);
        return false;
    }
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && global_ns() - t0 > limit) {
            atomicOr(err, 1u);
            return false;
        }
    }
}

// ------------------------------------------------------------------ symbol decoding
// ACGT without a table: for A=0x41, C=0x43, G=0x47, T=0x54 the two bits
// ((b >> 1) ^ (b >> 2)) & 3 are 0, 1, 2, 3. Works on four bytes at once; a
// byte is an ACGT letter iff the letter of its code equals the byte.
__device__ __forceinline__ uint32_t acgt_codes4(uint32_t w) { return ((w >> 1) ^ (w >> 2)) & 0x03030303u; }

__device__ __forceinline__ uint32_t acgt_mismatch4(uint32_t w, uint32_t codes) {
    uint32_t t = codes | (codes >> 4);                 // code k in nibble k (bytes 0,2 of t hold 2 nibbles each)
    uint32_t sel = __byte_perm(t, 0, 0x4420);          // nibbles c0 c1 c2 c3 in the low 16 bits
    uint32_t expect = __byte_perm(0x54474341u, 0, sel);  // "ACGT"[code] per byte
    return expect ^ w;                                 // 0 iff all four bytes are ACGT
}

// count a flagged entry (an output at the step) and remember the last one
template <uint32_t FLAGS>
__device__ __forceinline__ void track_flag(uint32_t v, uint32_t step, uint32_t &cnt, uint32_t &fv, uint32_t &fi) {
    const bool f = (v & FLAGS) != 0;
    cnt += f ? 1u : 0u;
    fv = f ? v : fv;
    fi = f ? step : fi;
}

// ------------------------------------------------------------------ table lookups
// Hybrid placement: one predicated pair, no branch. Lanes whose state lies in
// the shared-memory prefix read it there, the others read the full table
// through L2; a lane's word index is the same in both tables.
__device__ __forceinline__ uint32_t ld_hybrid(const uint32_t *stab, const uint32_t *gtab, uint32_t s,
                                              uint32_t smem_states, uint32_t idx, uint64_t pol) {
    uint32_t v;
    asm("{\n\t.reg .pred in_smem;\n\t.reg .u32 sa;\n\t.reg .u64 ga;\n\t"
        "setp.lt.u32 in_smem, %1, %2;\n\t"
        "mov.u32 %0, 0;\n\t"
        "mad.lo.u32 sa, %3, 4, %4;\n\t"
        "mad.wide.u32 ga, %3, 4, %5;\n\t"
        "@in_smem ld.shared.u32 %0, [sa];\n\t"
        "@!in_smem ld.global.nc.L2::cache_hint.u32 %0, [ga], %6;\n\t}"
        : "=r"(v)
        : "r"(s), "r"(smem_states), "r"(idx), "r"((uint32_t)__cvta_generic_to_shared(stab)), "l"(gtab), "l"(pol));
    return v;
}

// Hybrid placement with a 16-bit prefix (sigma = 4): a shared-memory entry is
// (next state << 1) | output bit; rotating it right by one bit gives the
// 32-bit form next | kFlag. The two predicated loads write separate
// registers (both start at zero, so an OR merges them).
__device__ __forceinline__ uint32_t ld_hybrid16(const uint32_t *stab, const uint32_t *gtab, uint32_t s,
                                                uint32_t smem_states, uint32_t idx, uint64_t pol) {
    uint32_t h = 0, g = 0;
    asm("{\n\t.reg .pred in_smem;\n\t.reg .u32 sa;\n\t.reg .u64 ga;\n\t"
        "setp.lt.u32 in_smem, %2, %3;\n\t"
        "mad.lo.u32 sa, %4, 2, %5;\n\t"
        "mad.wide.u32 ga, %4, 4, %6;\n\t"
        "@in_smem ld.shared.u16 %0, [sa];\n\t"
        "@!in_smem ld.global.nc.L2::cache_hint.u32 %1, [ga], %7;\n\t}"
        : "+r"(h), "+r"(g)
        : "r"(s), "r"(smem_states), "r"(idx), "r"((uint32_t)__cvta_generic_to_shared(stab)), "l"(gtab), "l"(pol));
    return g | __funnelshift_r(h, h, 1);
}

// MODE_OPT: the shared-memory prefix is a power of two of rows and the row
// index is masked into it, so the read is always in bounds; a state beyond
// the prefix reads a wrong entry, which the stage detects afterwards (the OR
// of the stage's entries has a bit at or above the prefix's size) and
// repairs by walking the stage again. smem_states is the prefix's row count.
template <int MODE>
__device__ __forceinline__ uint32_t lookup(const uint32_t *__restrict__ stab, const uint32_t *__restrict__ gtab,
                                           uint32_t smem_states, uint32_t sigma, uint32_t v, uint32_t c,
                                           uint64_t pol) {
    const uint32_t s = v & kStateMask;
    if (MODE == MODE_SMEM) return stab[s * sigma + c];
    if (MODE == MODE_OPT) return stab[(s & (smem_states - 1)) * sigma + c];
    if (MODE == MODE_H16) return ld_hybrid16(stab, gtab, s, smem_states, s * sigma + c, pol);
    return ld_hybrid(stab, gtab, s, smem_states, s * sigma + c, pol);
}

template <int MODE>
__device__ __forceinline__ uint32_t lookup4(const uint32_t *__restrict__ stab, const uint32_t *__restrict__ gtab,
                                            uint32_t smem_states, uint32_t v, uint32_t c, uint64_t pol) {
    // sigma = 4: index = s*4 + c; the shift drops the flag bit
    const uint32_t idx = (v << 2) | c;
    if (MODE == MODE_SMEM) return stab[idx];
    if (MODE == MODE_OPT) return stab[idx & (smem_states * 4u - 1u)];
    if (MODE == MODE_H16) return ld_hybrid16(stab, gtab, v & kStateMask, smem_states, idx, pol);
    return ld_hybrid(stab, gtab, v & kStateMask, smem_states, idx, pol);
}

// Two-symbol table (sigma = 4): index = s*16 + column, column = first symbol
// + 4 * second symbol; bits 31 and 30 of the entry are flags, not state bits.
template <int MODE>
__device__ __forceinline__ uint32_t lookup16(const uint32_t *__restrict__ stab, const uint32_t *__restrict__ gtab2,
                                             uint32_t smem_states, uint32_t v, uint32_t col, uint64_t pol) {
    const uint32_t s = v & kStateMask2;
    const uint32_t idx = (s << 4) | col;
    if (MODE == MODE_SMEM) return stab[idx];
    if (MODE == MODE_OPT) return stab[idx & (smem_states * 16u - 1u)];
    return ld_hybrid(stab, gtab2, s, smem_states, idx, pol);
}

// Emit the output of state `sid` at position `pos` for every lane with
// `has`; all 32 lanes must call this together.
__device__ __forceinline__ void emit_warp(bool has, uint32_t sid, uint64_t pos, uint64_t cbase,
                                          const SubsetDev &sd, const ScanParams &p, uint32_t lane) {
    unsigned m = __ballot_sync(kFull, has);
    if (m == 0) return;
    uint32_t b = 0, cnt = 0;
    if (has) {
        b = __ldg(sd.out_off + sid);
        cnt = __ldg(sd.out_off + sid + 1) - b;
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    uint32_t total = __shfl_sync(kFull, incl, 31);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(p.num, (unsigned long long)total);
    base = __shfl_sync(kFull, base, 0);
    unsigned long long slot = base + (incl - cnt);
    for (uint32_t t = 0; t < cnt; ++t) {
        uint32_t id = __ldg(sd.out_ids + b + t);
        if (slot + t < p.cap) p.keys[slot + t] = (pos << p.key_shift) | id;
        if (p.counts) atomicAdd(p.counts + cbase + id, 1ull);
    }
}

__device__ __forceinline__ uint32_t word_of(const uint4 &w, int e) {
    return e == 0 ? w.x : e == 1 ? w.y : e == 2 ? w.z : w.w;
}

// One stage of one chain walked symbol by symbol with every check (text
// edges, bytes outside the alphabet, table rows outside shared memory),
// emitting the output of every flagged state at main-stage positions. The
// stage's BX bytes are in w0 (and w1 when BX = 32) (every byte of the text inside the stage is
// there; positions before the text start reset the walk to the root). All 32
// lanes call it together; returns the state after the stage.
template <int FMT, int BX, bool H16>
__device__ __noinline__ uint32_t careful_walk(uint32_t s_in, int64_t pos0, bool active, bool main_stage,
                                             const uint4 w0, const uint4 w1, const ChainText &ct,
                                             const ScanParams &p, const SubsetDev &sd, const uint32_t *stab,
                                             const uint8_t *smap, uint32_t hot, uint32_t lane) {
    const uint32_t w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    constexpr int PER = (FMT == FMT_U8) ? 4 : 16;  // symbols per 32-bit word
    uint32_t sc = s_in;
    // the word index is static (unrolled), so the stage stays in registers
#pragma unroll
    for (int e = 0; e < BX / 4; ++e) {
        const uint32_t wv = w[e];
        for (int b = 0; b < PER; ++b) {
            const int64_t pos = pos0 + e * PER + b;
            const bool live = active && pos >= 0 && pos < (int64_t)ct.nsym;
            bool has = false;
            if (live) {
                const uint32_t c = (FMT == FMT_U8) ? (uint32_t)smap[(wv >> (8 * b)) & 0xffu] : (wv >> (2 * b)) & 3u;
                uint32_t nv = 0;
                if (c < p.sigma)
                    nv = lookup<H16 ? MODE_H16 : MODE_HYBRID>(stab, sd.table, hot, p.sigma, sc, c, l2_evict_last());
                sc = nv & kStateMask;
                has = main_stage && (nv & kFlag);
            } else if (pos < 0) {
                sc = 0;
            }
            emit_warp(has, sc, ct.vbase + (uint64_t)(pos < 0 ? 0 : pos), ct.cbase, sd, p, lane);
        }
    }
    return sc;
}

// The careful walk of a two-symbol-table scan: pairs of symbols through the
// two-symbol table (rows in shared memory as staged), the first symbol's
// state read from the one-symbol table only where it has an output; pairs
// at the text's end or holding a byte outside ACGT go symbol by symbol
// through the one-symbol table. Stage starts are even positions, so a pair
// never straddles the text start.
template <int FMT, int BX>
__device__ __noinline__ uint32_t careful_walk2(uint32_t s_in, int64_t pos0, bool active, bool main_stage,
                                              const uint4 w0, const uint4 w1, const ChainText &ct,
                                              const ScanParams &p, const SubsetDev &sd, const uint32_t *stab,
                                              const uint8_t *smap, uint32_t hot, uint32_t lane) {
    const uint32_t w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    constexpr int PER = (FMT == FMT_U8) ? 4 : 16;  // symbols per 32-bit word
    const uint64_t pol = l2_evict_last();
    uint32_t sc = s_in;
#pragma unroll
    for (int e = 0; e < BX / 4; ++e) {
        const uint32_t wv = w[e];
        for (int h = 0; h < PER / 2; ++h) {
            const int64_t pos = pos0 + e * PER + 2 * h;
            uint32_t c1, c2;
            if (FMT == FMT_U8) {
                c1 = smap[(wv >> (16 * h)) & 0xffu];
                c2 = smap[(wv >> (16 * h + 8)) & 0xffu];
            } else {
                c1 = (wv >> (4 * h)) & 3u;
                c2 = (wv >> (4 * h + 2)) & 3u;
            }
            const bool live1 = active && pos >= 0 && pos < (int64_t)ct.nsym;
            const bool live2 = active && pos + 1 >= 0 && pos + 1 < (int64_t)ct.nsym;
            bool has1 = false, has2 = false;
            uint32_t mid = 0;
            if (live1 && live2 && c1 < 4u && c2 < 4u) {
                const uint32_t nv = ld_hybrid(stab, sd.table2, sc, hot, (sc << 4) | c1 | (c2 << 2), pol);
                has1 = main_stage && (nv & kFlag1);
                has2 = main_stage && (nv & kFlag);
                if (has1) mid = ld_table(sd.table + ((uint64_t)sc << 2) + c1, pol) & kStateMask;
                sc = nv & kStateMask2;
            } else {
                if (live1) {
                    const uint32_t nv = c1 < 4u ? ld_table(sd.table + ((uint64_t)sc << 2) + c1, pol) : 0u;
                    mid = sc = nv & kStateMask;
                    has1 = main_stage && (nv & kFlag);
                } else if (pos < 0) {
                    sc = 0;
                }
                if (live2) {
                    const uint32_t nv = c2 < 4u ? ld_table(sd.table + ((uint64_t)sc << 2) + c2, pol) : 0u;
                    sc = nv & kStateMask;
                    has2 = main_stage && (nv & kFlag);
                } else if (pos + 1 < 0) {
                    sc = 0;
                }
            }
            emit_warp(has1, mid, ct.vbase + (uint64_t)(pos < 0 ? 0 : pos), ct.cbase, sd, p, lane);
            emit_warp(has2, sc, ct.vbase + (uint64_t)(pos + 1 < 0 ? 0 : pos + 1), ct.cbase, sd, p, lane);
        }
    }
    return sc;
}

// ------------------------------------------------------------------ the kernel
// Shared memory per warp and pipeline slot: C boxes of 32 rows x BX bytes
// (one per chain group, written by one 2-D TMA each) and one BX-byte slot
// for the ragged last row (written by a 1-D TMA), padded to 128 bytes.
__host__ __device__ constexpr uint32_t slot_bytes_for(uint32_t C, uint32_t BX) { return C * 32u * BX + 128u; }

// The chain's text: in single-text mode the row index is the text row; in
// batch mode the row's text is found by binary search over the items.
template <bool BATCH>
__device__ __forceinline__ bool chain_text(uint64_t row, const ScanParams &p, ChainText &ct) {
    if (!BATCH) {
        ct.row_in_text = row;
        ct.nsym = p.nsym;
        ct.vbase = 0;
        ct.cbase = 0;
        return row >= p.row_begin && row < p.row_end;
    }
    uint32_t lo = 0, hi = p.num_items;  // first item whose row_begin > row
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (p.items[mid].row_begin <= row) lo = mid + 1;
        else hi = mid;
    }
    if (lo == 0) return false;
    const BatchItemDev it = p.items[lo - 1];
    if (row >= it.row_begin + it.rows) return false;
    ct.row_in_text = row - it.row_begin;
    ct.nsym = it.nsym;
    ct.vbase = it.vbase;
    ct.cbase = it.cbase;
    return true;
}

template <int FMT, int ALPHA, int MODE, int BX, int C, bool BATCH, bool TRACK, int R>
__global__ void __launch_bounds__(512, 1)
    scan_kernel(const __grid_constant__ ScanParams p, const __grid_constant__ CUtensorMap rows_map,
                const __grid_constant__ CUtensorMap tail_map) {
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr uint32_t SYM_PER_STAGE = (FMT == FMT_U8) ? BX : BX * 4;
    constexpr uint32_t SLOT = slot_bytes_for(C, BX);
    constexpr uint32_t BOX = 32u * BX;  // bytes of one chain group's box
    // R = symbols per lookup: 1 (one-symbol table) or 2 (two-symbol table, sigma = 4)
    static_assert(R == 1 || (R == 2 && (FMT == FMT_P2 || ALPHA == ALPHA_ACGT)), "two-symbol table needs ACGT");
    constexpr uint32_t FLAGS = R == 2 ? (kFlag | kFlag1) : kFlag;
    constexpr uint32_t SMASK = R == 2 ? kStateMask2 : kStateMask;

    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t *stab = reinterpret_cast<uint32_t *>(smem);
    uint8_t *smap = smem + (((size_t)p.table_words * 4 + 127) & ~(size_t)127);
    uint8_t *stage = reinterpret_cast<uint8_t *>(((uintptr_t)(smap + 256) + 127) & ~(uintptr_t)127);
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage + (size_t)nwarps * kNS * SLOT);
    uint8_t *my_stage = stage + (size_t)warp * kNS * SLOT;
    uint64_t *my_bars = bars + warp * kNS;

    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) smap[i] = p.sym_of_byte[i];
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < nwarps * kNS; ++i) mbar_init(bars + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t parity = 0;  // bit i = parity of the phase slot i waits for next
    bool aborted = false;
    const uint64_t xpol = l2_evict_first();  // text
    const uint64_t tpol = l2_evict_last();   // goto table
    int cur_k = -1;
    const uint32_t sigma = p.sigma;
    const int64_t L = p.row_bytes;

    for (uint64_t tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
        uint32_t k;
        uint64_t tile_row0;
        if (BATCH) {
            const BatchTileDev td = p.tiles[tile];
            k = td.machine;
            tile_row0 = td.row0;
        } else {
            k = (uint32_t)(tile % p.K);
            tile_row0 = p.row_begin + (tile / p.K) * p.rows_per_tile;
        }
        const SubsetDev sd = p.subs[k];
        // rows staged in shared memory
        const uint32_t hot = min(MODE == MODE_H16 ? sd.rows16 : sd.states, p.smem_rows);
        // fast-loop lookups: MODE_OPT masks with the launch's power-of-two row
        // count (a smaller subset's states all lie below it, so its indices
        // pass the mask unchanged)
        const uint32_t lk = MODE == MODE_OPT ? p.smem_rows : hot;
        if ((int)k != cur_k) {
            __syncthreads();  // every warp is done with the previous table
            const uint32_t *src = MODE == MODE_H16 ? reinterpret_cast<const uint32_t *>(sd.table16)
                                  : R == 2          ? sd.table2
                                                    : sd.table;
            const uint32_t words = MODE == MODE_H16 ? hot * 2u : hot * (R == 2 ? 16u : sigma);
            const uint4 *src4 = reinterpret_cast<const uint4 *>(src);
            uint4 *dst4 = reinterpret_cast<uint4 *>(stab);
            for (uint32_t i = threadIdx.x; i < words / 4; i += blockDim.x) dst4[i] = __ldg(src4 + i);
            for (uint32_t i = (words & ~3u) + threadIdx.x; i < words; i += blockDim.x) stab[i] = __ldg(src + i);
            __syncthreads();
            cur_k = (int)k;
        }
        if (aborted) continue;  // keeps taking part in the CTA barriers above, does no work

        const uint32_t warm_bytes = (FMT == FMT_U8) ? sd.warm : (sd.warm + 3) / 4;
        const uint32_t nW = (warm_bytes + BX - 1) / BX;
        const uint32_t nst = nW + p.row_bytes / BX;
        const uint64_t row0 = tile_row0 + (uint64_t)warp * 32 * C;
        if (row0 >= p.row_end) continue;
        const bool tail_in_warp = !BATCH && p.tail_bytes && p.full_rows >= row0 && p.full_rows < row0 + 32 * C &&
                                  p.full_rows < p.row_end;

        // lane 0 issues one 2-D box per chain group (and the tail row's 1-D box)
        auto issue = [&](uint32_t s) {
            const uint32_t slot = s % kNS;
            uint8_t *base = my_stage + slot * SLOT;
            uint64_t *bar = my_bars + slot;
            const int64_t o = (int64_t)s * BX - (int64_t)nW * BX;  // byte offset from the row start
            const int64_t dy = o >= 0 ? o / L : -((-o + L - 1) / L);
            const int32_t col = (int32_t)(o - dy * L);
            uint32_t bytes = 0;
#pragma unroll
            for (int j = 0; j < C; ++j)
                if (row0 + (uint64_t)j * 32 < p.num_rows) bytes += BOX;
            const bool tail_now = tail_in_warp && o >= 0;
            if (tail_now) bytes += BX;
            mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
            for (int j = 0; j < C; ++j)
                if (row0 + (uint64_t)j * 32 < p.num_rows)
                    tma_load_2d(base + j * BOX, &rows_map, col, (int32_t)((int64_t)(row0 + j * 32) + dy), bar, xpol);
            if (tail_now) tma_load_1d(base + C * BOX, &tail_map, (int32_t)o, bar, xpol);
        };

        if (lane == 0)
            for (uint32_t s = 0; s < (uint32_t)kNS && s < nst; ++s) issue(s);

        uint64_t row[C];
        bool active[C];
        uint32_t st8[C];
        ChainText ct[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            row[j] = row0 + (uint64_t)j * 32 + lane;
            active[j] = chain_text<BATCH>(row[j], p, ct[j]);
            st8[j] = 0;
        }

        for (uint32_t s = 0; s < nst; ++s) {
            const uint32_t slot = s % kNS;
            if (!wait_phase(my_bars + slot, (parity >> slot) & 1u, p.err, p.wait_ns)) {
                aborted = true;
                break;
            }
            parity ^= 1u << slot;
            const int64_t o = (int64_t)s * BX - (int64_t)nW * BX;
            const bool main_stage = o >= 0;
            // this stage's BX bytes of every chain into registers, then refill the slot
            uint4 data[C][2];
            const uint8_t *base = my_stage + slot * SLOT;
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const bool tail_row = tail_in_warp && main_stage && row[j] == p.full_rows;
                const uint4 *b4 = reinterpret_cast<const uint4 *>(tail_row ? base + C * BOX : base + j * BOX + lane * BX);
                if (BX == 32) {
                    const uint32_t swz = (lane >> 2) & 1u;  // lanes l and l+4 read different halves first
                    const uint4 t0 = b4[swz], t1 = b4[swz ^ 1u];
                    data[j][0] = swz ? t1 : t0;
                    data[j][1] = swz ? t0 : t1;
                } else {
                    data[j][0] = b4[0];
                    data[j][1] = make_uint4(0, 0, 0, 0);
                }
            }
            __syncwarp();
            if (s + kNS < nst) {
                fence_proxy_async();
                if (lane == 0) issue(s + kNS);
            }

            int64_t pos0[C];
            bool fast[C], dead[C], before[C];
            uint32_t v[C], acc[C], bad[C], s_in[C];
            // flagged steps of each chain in this stage: how many, and the last
            // one (its entry and step), so a stage with one match emits it
            // without walking the stage again
            uint32_t fcnt[C], fv[C], fi[C];
#pragma unroll
            for (int j = 0; j < C; ++j) {
                fcnt[j] = 0;
                fv[j] = 0;
                fi[j] = 0;
                const int64_t b0 = (int64_t)ct[j].row_in_text * L + o;
                pos0[j] = (FMT == FMT_U8) ? b0 : b0 * 4;
                dead[j] = !active[j] || pos0[j] >= (int64_t)ct[j].nsym;
                before[j] = !dead[j] && pos0[j] + (int64_t)SYM_PER_STAGE <= 0;
                fast[j] = !dead[j] && pos0[j] >= 0 && pos0[j] + (int64_t)SYM_PER_STAGE <= (int64_t)ct[j].nsym;
                s_in[j] = st8[j];
                v[j] = s_in[j];
                acc[j] = 0;
                bad[j] = 0;
            }
            // The C chains advance together, one lookup each per round, so their
            // lookups are independent and overlap. Chains off the fast path walk
            // in-bounds garbage that is discarded.
            if constexpr (R == 2) {
                if constexpr (FMT == FMT_U8) {
#pragma unroll
                    for (int e = 0; e < (int)(BX / 4); ++e) {
                        uint32_t cw[C];
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            const uint32_t w = word_of(data[j][e >> 2], e & 3);
                            cw[j] = acgt_codes4(w);
                            bad[j] |= acgt_mismatch4(w, cw[j]);
                        }
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
#pragma unroll
                            for (int j = 0; j < C; ++j) {
                                // codes of bytes 2h and 2h+1 -> column c1 + 4*c2
                                const uint32_t col = ((cw[j] >> (16 * h)) & 3u) | ((cw[j] >> (16 * h + 6)) & 12u);
                                v[j] = lookup16<MODE>(stab, sd.table2, lk, v[j], col, tpol);
                                acc[j] |= v[j];
                                if constexpr (TRACK) track_flag<FLAGS>(v[j], e * 2 + h, fcnt[j], fv[j], fi[j]);
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < (int)(BX / 4); ++e) {
#pragma unroll
                        for (int h = 0; h < 8; ++h) {
#pragma unroll
                            for (int j = 0; j < C; ++j) {
                                // a nibble of packed text is the column (first symbol in its low bits)
                                const uint32_t col = (word_of(data[j][e >> 2], e & 3) >> (4 * h)) & 15u;
                                v[j] = lookup16<MODE>(stab, sd.table2, lk, v[j], col, tpol);
                                acc[j] |= v[j];
                                if constexpr (TRACK) track_flag<FLAGS>(v[j], e * 8 + h, fcnt[j], fv[j], fi[j]);
                            }
                        }
                    }
                }
            } else if (FMT == FMT_U8 && ALPHA == ALPHA_ACGT) {
#pragma unroll
                for (int e = 0; e < (int)(BX / 4); ++e) {
                    uint32_t cw[C];
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        const uint32_t w = word_of(data[j][e >> 2], e & 3);
                        cw[j] = acgt_codes4(w);
                        bad[j] |= acgt_mismatch4(w, cw[j]);
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            v[j] = lookup4<MODE>(stab, sd.table, lk, v[j], (cw[j] >> (8 * b)) & 3u, tpol);
                            acc[j] |= v[j];
                            if constexpr (TRACK) track_flag<kFlag>(v[j], e * 4 + b, fcnt[j], fv[j], fi[j]);
                        }
                    }
                }
            } else if (FMT == FMT_U8) {
#pragma unroll
                for (int e = 0; e < (int)(BX / 4); ++e) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            const uint32_t c = smap[(word_of(data[j][e >> 2], e & 3) >> (8 * b)) & 0xffu];
                            const uint32_t nv = lookup<MODE>(stab, sd.table, lk, sigma, v[j], c < sigma ? c : 0u, tpol);
                            v[j] = c < sigma ? nv : 0u;
                            acc[j] |= v[j];
                            if constexpr (TRACK) track_flag<kFlag>(v[j], e * 4 + b, fcnt[j], fv[j], fi[j]);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < (int)(BX / 4); ++e) {
#pragma unroll
                    for (int b = 0; b < 16; ++b) {
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            v[j] = lookup4<MODE>(stab, sd.table, lk, v[j], (word_of(data[j][e >> 2], e & 3) >> (2 * b)) & 3u,
                                          tpol);
                            acc[j] |= v[j];
                            if constexpr (TRACK) track_flag<kFlag>(v[j], e * 16 + b, fcnt[j], fv[j], fi[j]);
                        }
                    }
                }
            }
            // TRACK (template): the fast loop counted flagged steps, so a stage
            // with a single match emits it directly (pays off when matches are
            // frequent or the scan waits on L2 anyway); off, any flagged stage is
            // walked again (cheaper when the scan is issue-bound)
            bool need[C], single[C];
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if (fast[j]) st8[j] = v[j] & SMASK;
                else if (before[j]) st8[j] = 0;
                // with the two-symbol table a single flagged step is emitted
                // directly only when its output is at the second symbol
                const bool flagged = TRACK ? (fcnt[j] > 1 || (R == 2 && fcnt[j] == 1 && (fv[j] & kFlag1)))
                                           : (acc[j] & FLAGS) != 0;
                // MODE_OPT: a state at or beyond the prefix was looked up
                const bool outside = MODE == MODE_OPT && ((acc[j] | s_in[j]) & SMASK) >= lk;
                need[j] = !dead[j] && !before[j] && (!fast[j] || bad[j] != 0 || outside || (main_stage && flagged));
                single[j] = TRACK && !need[j] && fast[j] && main_stage && fcnt[j] == 1;
            }
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if (__any_sync(kFull, need[j])) {
                    // walked again by all lanes, emitting every flagged step of every lane
                    uint32_t sc;
                    if constexpr (R == 2)
                        sc = careful_walk2<FMT, BX>(s_in[j], pos0[j], active[j], main_stage, data[j][0], data[j][1],
                                                    ct[j], p, sd, stab, smap, hot, lane);
                    else
                        sc = careful_walk<FMT, BX, MODE == MODE_H16>(s_in[j], pos0[j], active[j], main_stage, data[j][0], data[j][1],
                                                   ct[j], p, sd, stab, smap, hot, lane);
                    if (!dead[j]) st8[j] = sc;
                } else if (__any_sync(kFull, single[j])) {
                    emit_warp(single[j], fv[j] & SMASK, ct[j].vbase + (uint64_t)(pos0[j] + R * fi[j] + (R - 1)),
                              ct[j].cbase, sd, p, lane);
                }
            }
        }
    }
    if (aborted && lane == 0) {
        // let copies already issued by this warp land before the CTA exits (bounded)
        for (uint32_t slot = 0; slot < (uint32_t)kNS; ++slot) {
            uint64_t t0 = global_ns();
            while (!mbar_try_wait(my_bars + slot, (parity >> slot) & 1u) && global_ns() - t0 < 100000000ull) {
            }
        }
    }
}

// ------------------------------------------------------------------ instantiation
using KernelFn = void (*)(ScanParams, CUtensorMap, CUtensorMap);

template <int FMT, int ALPHA, int MODE, bool BATCH, bool TRACK, int R>
KernelFn pick_shape(uint32_t bx, uint32_t C) {
    if (bx == 16)
        return C == 4 ? scan_kernel<FMT, ALPHA, MODE, 16, 4, BATCH, TRACK, R> : scan_kernel<FMT, ALPHA, MODE, 16, 2, BATCH, TRACK, R>;
    switch (C) {
        case 1: return scan_kernel<FMT, ALPHA, MODE, 32, 1, BATCH, TRACK, R>;
        case 2: return scan_kernel<FMT, ALPHA, MODE, 32, 2, BATCH, TRACK, R>;
        default: return scan_kernel<FMT, ALPHA, MODE, 32, 4, BATCH, TRACK, R>;
    }
}

// mode: MODE_SMEM, MODE_HYBRID, MODE_OPT or MODE_H16 (the last two
// instantiated for single-text, one-symbol launches with 2 or 4 chains; null
// otherwise)
template <int FMT, int ALPHA, bool BATCH, bool TRACK, int R = 1>
KernelFn pick_variant(int mode, uint32_t bx, uint32_t C) {
    if (mode == MODE_OPT || mode == MODE_H16) {
        if constexpr (!BATCH && R == 1) {
            if (mode == MODE_OPT) {
                if (C == 2) return bx == 16 ? scan_kernel<FMT, ALPHA, MODE_OPT, 16, 2, BATCH, TRACK, R>
                                            : scan_kernel<FMT, ALPHA, MODE_OPT, 32, 2, BATCH, TRACK, R>;
                if (C == 4) return bx == 16 ? scan_kernel<FMT, ALPHA, MODE_OPT, 16, 4, BATCH, TRACK, R>
                                            : scan_kernel<FMT, ALPHA, MODE_OPT, 32, 4, BATCH, TRACK, R>;
            } else {
                if (C == 2) return bx == 16 ? scan_kernel<FMT, ALPHA, MODE_H16, 16, 2, BATCH, TRACK, R>
                                            : scan_kernel<FMT, ALPHA, MODE_H16, 32, 2, BATCH, TRACK, R>;
                if (C == 4) return bx == 16 ? scan_kernel<FMT, ALPHA, MODE_H16, 16, 4, BATCH, TRACK, R>
                                            : scan_kernel<FMT, ALPHA, MODE_H16, 32, 4, BATCH, TRACK, R>;
            }
        }
        return nullptr;
    }
    return mode == MODE_HYBRID ? pick_shape<FMT, ALPHA, MODE_HYBRID, BATCH, TRACK, R>(bx, C)
                               : pick_shape<FMT, ALPHA, MODE_SMEM, BATCH, TRACK, R>(bx, C);
}

// defined in the scan_k_*.cu translation units (compiled in parallel)
#define AC_KERNEL_SET(name)                                                              \
    KernelFn kernels_##name##_single_plain(int mode, uint32_t bx, uint32_t C);       \
    KernelFn kernels_##name##_single_track(int mode, uint32_t bx, uint32_t C);       \
    KernelFn kernels_##name##_batch_plain(int mode, uint32_t bx, uint32_t C);        \
    KernelFn kernels_##name##_batch_track(int mode, uint32_t bx, uint32_t C);        \
    inline KernelFn kernels_##name(bool batch, bool track, int mode, uint32_t bx, uint32_t C) { \
        if (batch) return track ? kernels_##name##_batch_track(mode, bx, C) : kernels_##name##_batch_plain(mode, bx, C); \
        return track ? kernels_##name##_single_track(mode, bx, C) : kernels_##name##_single_plain(mode, bx, C); \
    }
AC_KERNEL_SET(u8_acgt)
AC_KERNEL_SET(u8_map)
AC_KERNEL_SET(packed)
#undef AC_KERNEL_SET
// two-symbol table (single-text launches)
KernelFn kernels_u8_acgt_single_plain_r2(int mode, uint32_t bx, uint32_t C);
KernelFn kernels_u8_acgt_single_track_r2(int mode, uint32_t bx, uint32_t C);
KernelFn kernels_packed_single_plain_r2(int mode, uint32_t bx, uint32_t C);
KernelFn kernels_packed_single_track_r2(int mode, uint32_t bx, uint32_t C);

}  // namespace kern
}  // namespace acgb
