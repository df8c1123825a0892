// The short-text scan: one thread per row of one to four 16-byte words, for
// texts too short to keep the GPU busy with the pipelined kernels' rows.
//
// It computes exactly what the lean and general kernels compute -- the
// folded AC-opt machine of Section III walked one symbol per lookup, the
// output of Section II.A reported at every flagged state, rows of the
// input-focused split (Section III) each preceded by a warm-up of longest
// pattern - 1 symbols walked from the root -- for one 4-letter machine.
//
// The pipelined kernels stage each chain's row through shared memory 16
// bytes at a time, so a launch costs one copy round trip per stage even when
// rows are a few stages long. Here every thread loads its whole window
// (warm-up words and row words, at most nine 16-byte words) straight into
// registers with vector loads issued while the table is staged; a launch
// is one memory round trip and one walk of (warm-up + row) symbols per
// thread, and every warp of the grid walks at once.
//
//  * SHORT_FULL: the whole table (next | output bit, 16 bytes a state)
//    copied into shared memory as it is.
//  * SHORT_E16: the escape-coded 16-bit breadth-first prefix in shared
//    memory (the lean kernel's LEAN_E16 table), the rest read through L2.
//
// Bytes are mapped to symbols through the machine's symbol map, so any
// 4-letter alphabet works; a byte outside the alphabet sends the walk to the
// root (Section II.A: no pattern contains it).
#include "ac_internal.h"
#include "scan_short.cuh"

namespace acgb {
namespace kern {

// Symbol i (0 <= i < 16 * symbols per byte) of a 16-byte word.
template <int FMT>
__device__ __forceinline__ uint32_t word_symbol(const uint4 &v, uint32_t i, const uint8_t *smap) {
    constexpr uint32_t PER = (FMT == FMT_U8) ? 4 : 16;  // symbols per 32-bit word
    const uint32_t e = i / PER, b = i % PER;
    const uint32_t x = e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
    return (FMT == FMT_U8) ? (uint32_t)smap[(x >> (8 * b)) & 0xffu] : (x >> (2 * b)) & 3u;
}

// One lookup: the entry (next | output bit) of state s on symbol c; the root
// for a symbol outside the alphabet.
template <int SM>
__device__ __forceinline__ uint32_t short_step(uint32_t s, uint32_t c, const uint8_t *tab, uint32_t hot,
                                               const uint32_t *gtab) {
    if (c >= 4u) return 0u;
    if (SM == SHORT_FULL) return reinterpret_cast<const uint32_t *>(tab)[s * 4u + c];
    uint32_t nv = kEsc16;
    if (s < hot) nv = reinterpret_cast<const uint16_t *>(tab)[s * 4u + c];
    if (nv == kEsc16) nv = __ldg(gtab + (size_t)s * 4u + c);
    return nv;
}

__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

// E16 lookup (as the lean kernel's): the 16-bit prefix entry at shared
// address sa when s < hot and it is not the escape, else the 32-bit table
// entry at byte offset 2 * gi.
__device__ __forceinline__ uint32_t short_e16(uint32_t s, uint32_t sa, uint32_t gi, uint32_t hot,
                                              const uint32_t *gtab) {
    uint32_t e;
    asm("{\n\t.reg .pred ps, pg;\n\t.reg .u64 ga;\n\t"
        "setp.lt.u32 ps, %1, %3;\n\t"
        "mov.u32 %0, 65535;\n\t"
        "@ps ld.shared.u16 %0, [%2];\n\t"
        "setp.eq.u32 pg, %0, 65535;\n\t"
        "mad.wide.u32 ga, %4, 2, %5;\n\t"
        "@pg ld.global.nc.u32 %0, [ga];\n\t}"
        : "=r"(e)
        : "r"(s), "r"(sa), "r"(hot), "r"(gi), "l"(gtab));
    return e;
}

// One 16-byte word of symbols walked without any per-symbol check: every
// symbol lies inside the text and in the alphabet (ACGT bytes, or packed
// codes). FULL: the 32-bit table, entry at byte (s << 4) + 4c; E16: the
// 16-bit prefix (byte (s << 3) + 2c) and the 32-bit table beyond it. The
// state is updated in place; returns the OR of the entries (output flags).
template <int FMT, int SM>
__device__ __forceinline__ uint32_t short_fast_word(const uint4 &v, uint32_t &s, uint32_t sbase, uint32_t hot,
                                                    const uint32_t *gtab) {
    constexpr uint32_t SH = (SM == SHORT_FULL) ? 2 : 1;  // code -> byte offset in the row
    uint32_t acc = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint32_t x = e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
        constexpr int PER = (FMT == FMT_U8) ? 4 : 16;
        const uint32_t cw = (FMT == FMT_U8) ? (acgt_codes4(x) << SH) : x;
#pragma unroll
        for (int b = 0; b < PER; ++b) {
            uint32_t off;  // code << SH
            if (FMT == FMT_U8) off = __byte_perm(cw, 0, 0x4440 + b);
            else off = ((2 * b >= (int)SH) ? (cw >> (2 * b - SH)) : (cw << (SH - 2 * b))) & (3u << SH);
            uint32_t nv;
            if (SM == SHORT_FULL) {
                nv = lds_u32(sbase + (s << 4) + off);
            } else {
                const uint32_t gi = (s << 3) + off;
                nv = short_e16(s, sbase + gi, gi, hot, gtab);
            }
            acc |= nv;
            s = nv & kStateMask;
        }
    }
    return acc;
}

// The outputs of one row word per lane (has: the word is wholly inside the
// text and, for bytes, wholly A/C/G/T, and its walk met a flagged state):
// the word walked again from s_in, counting the outputs and keeping the last
// four flagged steps in registers (state << 6 | step; machines of fewer than
// 2^26 states), then one slot reservation for the whole warp and the keys
// written from those records; a lane with more than four flagged steps (or a
// larger machine) makes the warp walk the word once more to write.
// pos0: position of the word's first symbol. ooff / oids: the output offsets
// and ids. All 32 lanes call it together.
template <int FMT, int SM>
__device__ __forceinline__ void short_emit_word(bool has, const uint4 &v, uint32_t s_in, uint64_t pos0,
                                                uint32_t sbase, uint32_t hot, const uint32_t *gtab,
                                                const uint32_t *ooff, const uint32_t *oids, const ScanParams &p,
                                                uint32_t lane) {
    constexpr uint32_t SH = (SM == SHORT_FULL) ? 2 : 1;  // code -> byte offset in the row
    constexpr int PER = (FMT == FMT_U8) ? 4 : 16;        // symbols per 32-bit word
    auto step = [&](uint32_t s, uint32_t cw, int b) -> uint32_t {
        uint32_t off;
        if (FMT == FMT_U8) off = __byte_perm(cw, 0, 0x4440 + b);
        else off = ((2 * b >= (int)SH) ? (cw >> (2 * b - SH)) : (cw << (SH - 2 * b))) & (3u << SH);
        if (SM == SHORT_FULL) return lds_u32(sbase + (s << 4) + off);
        const uint32_t gi = (s << 3) + off;
        return short_e16(s, sbase + gi, gi, hot, gtab);
    };
    uint32_t cnt = 0, nrec = 0;
    uint32_t r0 = 0, r1 = 0, r2 = 0, r3 = 0;  // newest first
    if (has) {
        uint32_t s = s_in;
#pragma unroll 1
        for (int e = 0; e < 4; ++e) {
            const uint32_t x = word_of(v, e);
            const uint32_t cw = (FMT == FMT_U8) ? (acgt_codes4(x) << SH) : x;
#pragma unroll
            for (int b = 0; b < PER; ++b) {
                const uint32_t nv = step(s, cw, b);
                s = nv & kStateMask;
                if (nv & kFlag) {
                    cnt += ooff[s + 1] - ooff[s];
                    r3 = r2; r2 = r1; r1 = r0; r0 = (s << 6) | (uint32_t)(e * PER + b);
                    ++nrec;
                }
            }
        }
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(p.num, (unsigned long long)total);
    unsigned long long slot = __shfl_sync(kFull, base, 0) + (incl - cnt);
    auto write = [&](uint32_t st, uint32_t k) {
        const uint64_t pos = pos0 + k;
        const uint32_t o0 = ooff[st], o1 = ooff[st + 1];
        for (uint32_t t = o0; t < o1; ++t, ++slot) {
            const uint32_t id = oids[t];
            if (slot < p.cap) p.keys[slot] = (pos << p.key_shift) | id;
            if (p.counts) atomicAdd(p.counts + id, 1ull);
        }
    };
    if (!__any_sync(kFull, nrec > 4) && p.sub0.states < (1u << 26)) {
        if (nrec > 0) write(r0 >> 6, r0 & 63u);
        if (nrec > 1) write(r1 >> 6, r1 & 63u);
        if (nrec > 2) write(r2 >> 6, r2 & 63u);
        if (nrec > 3) write(r3 >> 6, r3 & 63u);
        return;
    }
    // some lane has more flagged steps than it kept: walk again and write
    if (has) {
        uint32_t s = s_in;
#pragma unroll 1
        for (int e = 0; e < 4; ++e) {
            const uint32_t x = word_of(v, e);
            const uint32_t cw = (FMT == FMT_U8) ? (acgt_codes4(x) << SH) : x;
#pragma unroll
            for (int b = 0; b < PER; ++b) {
                const uint32_t nv = step(s, cw, b);
                s = nv & kStateMask;
                if (nv & kFlag) write(s, (uint32_t)(e * PER + b));
            }
        }
    }
}

// all 16 bytes of the word are A, C, G or T
__device__ __forceinline__ bool word_is_acgt(const uint4 &v) {
    return (acgt_mismatch4(v.x, acgt_codes4(v.x)) | acgt_mismatch4(v.y, acgt_codes4(v.y)) |
            acgt_mismatch4(v.z, acgt_codes4(v.z)) | acgt_mismatch4(v.w, acgt_codes4(v.w))) == 0;
}

// MAXW: words of the window a thread holds (warm-up + row words <= MAXW).
// ACGT: byte text over exactly A, C, G, T (decoded without the symbol map).
template <int FMT, int SM, int MAXW, bool ACGT>
__global__ void __launch_bounds__(1024, 1) short_kernel(const __grid_constant__ ScanParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    pdl_release();  // the sort behind this launch may start; it waits for these results
    const SubsetDev &sd = p.sub0;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t warm_bytes = (FMT == FMT_U8) ? sd.warm : (sd.warm + 3) / 4;
    const uint32_t nw_warm = (warm_bytes + 15) / 16;
    const uint32_t nw = nw_warm + p.row_bytes / 16;  // <= MAXW (host-checked)
    const uint64_t row = p.row_begin + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = row < p.row_end;
    const int64_t nbytes = (int64_t)p.nbytes;
    const int64_t b0 = (int64_t)row * p.row_bytes - 16 * (int64_t)nw_warm;  // first byte of the window

    // The table (and the symbol map) into shared memory.
    const uint32_t tbytes = (SM == SHORT_FULL) ? sd.states * 16u : p.smem_rows * 8u;
    uint8_t *tab = smem;
    uint8_t *smap = smem + ((tbytes + 15) & ~15u);
    {
        const uint4 *src = (SM == SHORT_FULL) ? reinterpret_cast<const uint4 *>(sd.table)
                                              : reinterpret_cast<const uint4 *>(sd.table_e16);
        // asynchronous 16-byte copies: no registers held, every copy of the
        // thread in flight at once
        const uint32_t n16 = tbytes / 16;
        const uint32_t dst0 = smem_addr(tab);
        for (uint32_t i = threadIdx.x; i < n16; i += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst0 + 16 * i), "l"(src + i) : "memory");
        if ((tbytes & 15) && threadIdx.x == 0)  // an odd row count of the 16-bit prefix: its last 8 bytes
            *reinterpret_cast<uint2 *>(tab + (tbytes & ~15u)) =
                __ldg(reinterpret_cast<const uint2 *>(reinterpret_cast<const uint8_t *>(src) + (tbytes & ~15u)));
        for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) smap[i] = p.sym_of_byte[i];
    }
    // The launch before this one (the zeroing of the counter and counts, which
    // itself waited for everything before it) has finished from here on: the
    // text, written before the call, may be read and the outputs written.
    pdl_wait();

    // The window into registers; the loads overlap the table's copies.
    uint4 w[MAXW];
#pragma unroll
    for (int k = 0; k < MAXW; ++k) {
        w[k] = make_uint4(0, 0, 0, 0);
        const int64_t b = b0 + 16 * (int64_t)k;
        if (active && (uint32_t)k < nw) {
            if (b >= 0 && b + 16 <= nbytes) {
                w[k] = __ldg(reinterpret_cast<const uint4 *>(p.text + b));  // 16-byte aligned
            } else if (b + 16 > 0 && b < nbytes) {  // a text edge inside the word
                uint32_t v[4] = {0, 0, 0, 0};
                for (int j = 0; j < 16; ++j)
                    if (b + j >= 0 && b + j < nbytes) v[j >> 2] |= (uint32_t)__ldg(p.text + b + j) << (8 * (j & 3));
                w[k] = make_uint4(v[0], v[1], v[2], v[3]);
            }
        }
    }

    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const uint32_t *ooff = sd.out_off;
    const uint32_t *oids = sd.out_ids;

    // The walk, one word at a time (the window shifts down one word per
    // step): warm-up words from the root (positions before the text start
    // keep it there), then the row's words. A row word in which some lane of
    // the warp meets a flagged state is walked again by the warp, symbol by
    // symbol, emitting the outputs.
    const uint32_t hot = p.smem_rows;
    constexpr uint32_t SYM = (FMT == FMT_U8) ? 16 : 64;  // symbols per word
    const int64_t nsym = (int64_t)p.nsym;
    uint32_t s = 0;
#pragma unroll 1
    for (uint32_t k = 0; k < nw; ++k) {
        const uint4 cur = w[0];
#pragma unroll
        for (int j = 0; j + 1 < MAXW; ++j) w[j] = w[j + 1];
        const int64_t pos0 = (b0 + 16 * (int64_t)k) * (SYM / 16);
        const uint32_t s_in = s;
        uint32_t acc = 0;
        // a word wholly inside the text (and, for bytes, wholly A/C/G/T) is
        // walked without per-symbol checks
        const bool fast = active && pos0 >= 0 && pos0 + (int64_t)SYM <= nsym &&
                          (FMT == FMT_P2 || (ACGT && word_is_acgt(cur)));
        if (fast) {
            acc = short_fast_word<FMT, SM>(cur, s, smem_addr(tab), hot, sd.table);
        } else {
            // 16 symbols per inner pass: one pass for bytes, four for packed text
#pragma unroll 1
            for (uint32_t q = 0; q < SYM; q += 16) {
#pragma unroll
                for (uint32_t i = 0; i < 16; ++i) {
                    const int64_t pos = pos0 + q + i;
                    const uint32_t nv = short_step<SM>(s, word_symbol<FMT>(cur, q + i, smap), tab, hot, sd.table);
                    const bool live = active && pos >= 0 && pos < nsym;
                    s = live ? (nv & kStateMask) : 0u;
                    acc |= live ? nv : 0u;
                }
            }
        }
        if (k >= nw_warm) {
            // flagged words on the fast path: one walk and one reservation
            // per warp; words at a text edge or holding other bytes (rare):
            // symbol by symbol with every check
            const bool flagged = (acc & kFlag) != 0;
            if (__any_sync(kFull, fast && flagged))
                short_emit_word<FMT, SM>(fast && flagged, cur, s_in, (uint64_t)(pos0 < 0 ? 0 : pos0), smem_addr(tab),
                                         hot, sd.table, ooff, oids, p, lane);
            const bool hard = !fast && flagged;
            if (__any_sync(kFull, hard)) {
                uint32_t sc = s_in;
#pragma unroll 1
                for (uint32_t i = 0; i < SYM; ++i) {
                    const int64_t pos = pos0 + i;
                    const uint32_t nv = short_step<SM>(sc, word_symbol<FMT>(cur, i, smap), tab, hot, sd.table);
                    const bool live = active && pos >= 0 && pos < nsym;
                    sc = live ? (nv & kStateMask) : 0u;
                    emit_warp(hard && live && (nv & kFlag), sc, (uint64_t)(pos < 0 ? 0 : pos), 0, sd, p, lane);
                }
            }
        }
    }
}

template <int FMT, int SM, bool ACGT>
ShortFn pick_short(uint32_t words) {
    return words <= 5 ? short_kernel<FMT, SM, 5, ACGT> : short_kernel<FMT, SM, kShortMaxWords, ACGT>;
}

ShortFn short_u8_full(uint32_t words, bool acgt) {
    return acgt ? pick_short<FMT_U8, SHORT_FULL, true>(words) : pick_short<FMT_U8, SHORT_FULL, false>(words);
}
ShortFn short_u8_e16(uint32_t words, bool acgt) {
    return acgt ? pick_short<FMT_U8, SHORT_E16, true>(words) : pick_short<FMT_U8, SHORT_E16, false>(words);
}
ShortFn short_packed_full(uint32_t words) { return pick_short<FMT_P2, SHORT_FULL, false>(words); }
ShortFn short_packed_e16(uint32_t words) { return pick_short<FMT_P2, SHORT_E16, false>(words); }

}  // namespace kern
}  // namespace acgb
