// The lean scan: one-symbol tables of a 4-letter machine over ACGT bytes or
// 2-bit packed text, one text per launch.
//
// It computes exactly what scan_kernel computes (the folded AC-opt machine of
// Section III walked one symbol at a time, Section II.A's output at every
// flagged state; input-focused rows with a warm-up of longest pattern - 1
// symbols, pattern-focused subsets as tiles), with a fast loop cut down to a
// few instructions per symbol so that more chains fit on an SM:
//
//  * LEAN_SMEM32 (every row of the subset in shared memory): a shared-memory
//    entry is the byte offset of the next state's row (next << 4) with the
//    output bit in bit 0, so the next address is (entry & ~15) | 4*symbol --
//    one logic instruction, one shared load, one OR into the stage's
//    accumulator per symbol.
//  * LEAN_E16 (larger machines): a breadth-first prefix of 16-bit entries in
//    shared memory holding the next state itself, or an escape code when that
//    state has an output or does not fit 16 bits; a lookup is one predicated
//    shared load (state inside the prefix), then one predicated load of the
//    32-bit table through L2 (state beyond the prefix, or an escape). The
//    32-bit entry carries the output bit (bit 31), which the stage's OR
//    accumulator collects.
//
// Text staging is the same tensor-map TMA pipeline as scan_kernel with one
// slot per warp (the slot is refilled as soon as the lanes hold the stage in
// registers, and a stage of lookups takes far longer than the copy), so the
// staging costs 16 bytes of shared memory per chain. A stage whose
// accumulator shows an output (or that holds a byte outside ACGT, or touches
// a text edge) is walked again symbol by symbol by the whole warp
// (lean_careful) and its matches are emitted through emit_warp.
#pragma once

#include "scan_kernel.cuh"

namespace acgb {
namespace kern {

enum { LEAN_SMEM32 = kLeanSmem32, LEAN_E16 = kLeanE16 };
constexpr uint32_t kLeanBX = 16;  // text bytes per chain per stage

__host__ __device__ constexpr uint32_t lean_slot_bytes(uint32_t C) { return C * 32u * kLeanBX + 128u; }

// shared memory of a lean CTA besides the table: byte map, one staging slot
// and one mbarrier per warp, the table's mbarrier and state word, alignment
__host__ __device__ constexpr uint32_t lean_stage_bytes(uint32_t threads, uint32_t C) {
    return 256u + 128u + 128u + 16u + (threads / 32u) * (lean_slot_bytes(C) + 8u);
}

// E16 lookup of entry (state u, symbol): sa = its shared address in the 16-bit
// prefix (read only when u < hot, i.e. u is a prefix row without the output
// bit), gi = its byte offset there (the 32-bit table's byte offset is twice
// that). An escape, or a state beyond the prefix, reads the 32-bit table.
// Returns the next entry: a state id (16-bit prefix) or a 32-bit table entry
// (state id | kFlag when its output is not empty).
__device__ __forceinline__ uint32_t e16_step(uint32_t u, uint32_t sa, uint32_t gi, uint32_t hot,
                                             const uint32_t *gtab) {
    uint32_t e;
    asm("{\n\t.reg .pred ps, pg;\n\t.reg .u64 ga;\n\t"
        "setp.lt.u32 ps, %1, %3;\n\t"
        "mov.u32 %0, 65535;\n\t"
        "@ps ld.shared.u16 %0, [%2];\n\t"
        "setp.eq.u32 pg, %0, 65535;\n\t"
        "mad.wide.u32 ga, %4, 2, %5;\n\t"
        "@pg ld.global.nc.L1::no_allocate.u32 %0, [ga];\n\t}"
        : "=r"(e)
        : "r"(u), "r"(sa), "r"(hot), "r"(gi), "l"(gtab));
    return e;
}

// The text pipeline with 32-bit shared-window addresses (fewer registers than
// generic pointers).
__device__ __forceinline__ void mbar_expect_s(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait_s(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: false (and the error word set) once
// `limit` ns have passed; a limit of 0 gives up before the first check.
__device__ __forceinline__ bool wait_phase_s(uint32_t bar, uint32_t parity, uint32_t *err, uint64_t limit) {
    if (limit == 0) {
        atomicOr(err, 1u);
        return false;
    }
    if (mbar_try_wait_s(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_s(bar, parity)) return true;
        if ((it & 255u) == 0 && global_ns() - t0 > limit) {
            atomicOr(err, 1u);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_2d_s(uint32_t dst, const CUtensorMap *map, int32_t x, int32_t y, uint32_t bar,
                                         uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void tma_1d_s(uint32_t dst, const CUtensorMap *map, int32_t x, uint32_t bar,
                                         uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2}], [%3], %4;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(bar), "l"(pol)
        : "memory");
}

__device__ __forceinline__ uint2 lds64(uint32_t a) {
    uint2 v;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a) : "memory");
    return v;
}

__device__ __forceinline__ uint4 lds128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a)
                 : "memory");
    return v;
}

// Next state of clean state s on symbol c (< 4) in the 32-bit entry format
// (next | kFlag when its output is not empty), for the careful walk.
template <int LM>
__device__ __forceinline__ uint32_t lean_lookup(const uint8_t *tab, uint32_t hot, const uint32_t *gtab,
                                                uint32_t s, uint32_t c, uint64_t pol) {
    if (LM == LEAN_SMEM32) {
        const uint32_t e = reinterpret_cast<const uint32_t *>(tab)[s * 4u + c];
        return (e >> 4) | (e << 31);
    } else {
        if (s < hot) {
            const uint32_t e = reinterpret_cast<const uint16_t *>(tab)[s * 4u + c];
            if (e != kEsc16) return e;
        }
        return ld_table(gtab + (size_t)s * 4u + c, pol);
    }
}

// One stage of one chain walked symbol by symbol with every check (text
// edges, bytes outside ACGT), emitting the output of every flagged state at
// main-stage positions. The stage's 16 bytes (row `row`, byte offset o from
// the row start; negative in the warm-up) are read again from global memory:
// the staging slot has been refilled by then, and this path is rare. s_in is
// a clean state id; returns the clean state after the stage. All 32 lanes
// call it together. Inlined at a single site of the kernel (a call would make
// the kernel keep its registers in local memory around it).
template <int FMT, int LM>
__device__ __forceinline__ uint32_t lean_careful(uint32_t s_in, uint64_t row, int64_t o, bool main_stage,
                                             const ScanParams &p, const SubsetDev *sdp, const uint8_t *tab,
                                             const uint8_t *smap, uint32_t hot, uint32_t lane) {
    const SubsetDev &sd = *sdp;
    const bool active = row >= p.row_begin && row < p.row_end;
    const int64_t b0 = (int64_t)row * (int64_t)p.row_bytes + o;  // byte offset of the stage in the text
    uint32_t w[4] = {0, 0, 0, 0};
    if (active) {
        if (b0 >= 0 && b0 + 16 <= (int64_t)p.nbytes) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p.text + b0));  // 16-byte aligned
            w[0] = v.x;
            w[1] = v.y;
            w[2] = v.z;
            w[3] = v.w;
        } else {
            for (int k = 0; k < 16; ++k)
                if (b0 + k >= 0 && b0 + k < (int64_t)p.nbytes) w[k >> 2] |= (uint32_t)__ldg(p.text + b0 + k) << (8 * (k & 3));
        }
    }
    constexpr int PER = (FMT == FMT_U8) ? 4 : 16;
    const int64_t pos0 = (FMT == FMT_U8) ? b0 : b0 * 4;
    const uint64_t pol = l2_evict_last();
    const int64_t nsym = (int64_t)p.nsym;
    uint32_t sc = s_in;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint32_t wv = w[e];
#pragma unroll 1
        for (int b = 0; b < PER; ++b) {
            const int64_t pos = pos0 + e * PER + b;
            const bool live = active && pos >= 0 && pos < nsym;
            bool has = false;
            if (live) {
                const uint32_t c = (FMT == FMT_U8) ? (uint32_t)smap[(wv >> (8 * b)) & 0xffu] : (wv >> (2 * b)) & 3u;
                const uint32_t nv = c < 4u ? lean_lookup<LM>(tab, hot, sd.table, sc, c, pol) : 0u;
                sc = nv & kStateMask;
                has = main_stage && (nv & kFlag);
            } else if (pos < 0) {
                sc = 0;
            }
            emit_warp(has, sc, (uint64_t)(pos < 0 ? 0 : pos), 0, sd, p, lane);
        }
    }
    return sc;
}

// The matches of one queued stage per lane (has): the stage's 16 bytes (all
// A/C/G/T or packed codes, every position inside the text and owned by its
// row, at byte b0) walked again from s_in, counting the outputs and keeping
// the last four flagged (state, step) pairs in registers; then one slot
// reservation for the whole warp and the keys written from those pairs
// (one dependent walk and one atomic round trip per warp). A lane with more
// than four flagged steps makes the warp walk again to write. All 32 lanes
// call it together.
template <int FMT, int LM>
__device__ __forceinline__ void lean_emit_stage(bool has, uint32_t s_in, uint64_t b0, const ScanParams &p,
                                                const SubsetDev &sd, const uint8_t *tab, uint32_t hot,
                                                uint32_t lane) {
    constexpr int PER = (FMT == FMT_U8) ? 4 : 16;  // symbols per 32-bit word
    uint32_t w[4] = {0, 0, 0, 0};
    if (has) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p.text + b0));  // 16-byte aligned
        w[0] = (FMT == FMT_U8) ? acgt_codes4(v.x) : v.x;
        w[1] = (FMT == FMT_U8) ? acgt_codes4(v.y) : v.y;
        w[2] = (FMT == FMT_U8) ? acgt_codes4(v.z) : v.z;
        w[3] = (FMT == FMT_U8) ? acgt_codes4(v.w) : v.w;
    }
    const uint64_t pol = l2_evict_last();
    const uint64_t pos0 = (FMT == FMT_U8) ? b0 : b0 * 4;
    uint32_t cnt = 0, nrec = 0;
    uint32_t rs0 = 0, rs1 = 0, rs2 = 0, rs3 = 0, rp0 = 0, rp1 = 0, rp2 = 0, rp3 = 0;  // newest first
    {
        uint32_t sc = s_in;
#pragma unroll 1
        for (int e = 0; e < 4; ++e) {
#pragma unroll 4
            for (int b = 0; b < PER; ++b) {
                const uint32_t c = (FMT == FMT_U8) ? (w[e] >> (8 * b)) & 3u : (w[e] >> (2 * b)) & 3u;
                const uint32_t nv = has ? lean_lookup<LM>(tab, hot, sd.table, sc, c, pol) : 0u;
                sc = nv & kStateMask;
                if (nv & kFlag) {
                    cnt += __ldg(sd.out_off + sc + 1) - __ldg(sd.out_off + sc);
                    rs3 = rs2; rs2 = rs1; rs1 = rs0; rs0 = sc;
                    rp3 = rp2; rp2 = rp1; rp1 = rp0; rp0 = (uint32_t)(e * PER + b);
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
    auto write = [&](uint32_t st, uint32_t step) {
        const uint64_t pos = pos0 + step;
        const uint32_t o0 = __ldg(sd.out_off + st), o1 = __ldg(sd.out_off + st + 1);
        for (uint32_t t = o0; t < o1; ++t, ++slot) {
            const uint32_t id = __ldg(sd.out_ids + t);
            if (slot < p.cap) p.keys[slot] = (pos << p.key_shift) | id;
            if (p.counts) atomicAdd(p.counts + id, 1ull);
        }
    };
    if (!__any_sync(kFull, nrec > 4)) {
        if (nrec > 0) write(rs0, rp0);
        if (nrec > 1) write(rs1, rp1);
        if (nrec > 2) write(rs2, rp2);
        if (nrec > 3) write(rs3, rp3);
        return;
    }
    // some lane has more flagged steps than it kept: walk again and write
    uint32_t sc = s_in;
#pragma unroll 1
    for (int e = 0; e < 4; ++e) {
#pragma unroll 4
        for (int b = 0; b < PER; ++b) {
            const uint32_t c = (FMT == FMT_U8) ? (w[e] >> (8 * b)) & 3u : (w[e] >> (2 * b)) & 3u;
            const uint32_t nv = has ? lean_lookup<LM>(tab, hot, sd.table, sc, c, pol) : 0u;
            sc = nv & kStateMask;
            if (nv & kFlag) write(sc, (uint32_t)(e * PER + b));
        }
    }
}

// symbol code of 2-bit packed symbol b of word w, times 2 (E16) or 4 (SMEM32)
template <int SH>
__device__ __forceinline__ uint32_t packed_code(uint32_t w, int b) {
    // code << SH = bits [2b, 2b+2) of w moved to [SH, SH+2)
    return (2 * b >= SH ? (w >> (2 * b - SH)) : (w << (SH - 2 * b))) & (3u << SH);
}

template <int FMT, int LM, int C, int NT>
__global__ void __launch_bounds__(NT, 1)
    lean_kernel(const __grid_constant__ ScanParams p, const __grid_constant__ CUtensorMap rows_map,
                const __grid_constant__ CUtensorMap tail_map) {
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr uint32_t BX = kLeanBX;
    constexpr uint32_t SYM = (FMT == FMT_U8) ? BX : BX * 4;  // symbols per stage
    constexpr uint32_t SLOT = lean_slot_bytes(C);
    constexpr uint32_t BOX = 32u * BX;
    constexpr uint32_t FLAG = LM == LEAN_SMEM32 ? 1u : kFlag;

    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint8_t *tab = smem;
    uint8_t *smap = smem + (((size_t)p.table_words * 4 + 127) & ~(size_t)127);
    uint8_t *stage = reinterpret_cast<uint8_t *>(((uintptr_t)(smap + 256) + 127) & ~(uintptr_t)127);
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage + (size_t)nwarps * SLOT);
    const uint32_t my_stage = smem_addr(stage) + warp * SLOT;  // shared-window addresses
    const uint32_t my_bar = smem_addr(bars + warp);
    uint64_t *tbars = bars + nwarps;  // the table's mbarrier, then its state word

    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) smap[i] = p.sym_of_byte[i];
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i <= nwarps; ++i) mbar_init(bars + i, 1);  // one per warp, one for the table
        // table copy state: [0] = the last copy landed, [1] = barrier phase | (a copy is late) << 1
        reinterpret_cast<uint32_t *>(tbars + 1)[0] = 1;
        reinterpret_cast<uint32_t *>(tbars + 1)[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t parity = 0;
    bool aborted = false;
    const uint64_t xpol = l2_evict_first();  // text
    const uint32_t sbase = smem_addr(tab);
    const int64_t nsym = (int64_t)p.nsym;

    // Stage subset k's table into shared memory (all threads of the CTA).
    // Stage subset k's table into shared memory (all threads of the CTA). The
    // escape-coded prefix is copied as it is by one bulk copy (the TMA engine
    // streams it); the row-offset table is converted on the way, eight
    // independent loads per thread in flight.
    // (the table copy's state lives in shared memory, not in registers the scan loop would carry)
    auto stage_table = [&](const SubsetDev *sdp, uint32_t hot) {
        __syncthreads();  // every warp is done with the previous table
        if (LM == LEAN_SMEM32) {
            // entry -> (next << 4) | output bit: the byte offset of the next row
            const uint32_t words = hot * 4u;
            const uint32_t *gtab = sdp->table;
            uint32_t *t32 = reinterpret_cast<uint32_t *>(tab);
            for (uint32_t base = threadIdx.x; base < words; base += blockDim.x * 8) {
                uint32_t v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t i = base + k * blockDim.x;
                    v[k] = i < words ? __ldg(gtab + i) : 0u;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t i = base + k * blockDim.x;
                    if (i < words) t32[i] = ((v[k] & kStateMask) << 4) | (v[k] >> 31);
                }
            }
        } else {
            const uint32_t bytes = hot * 8u;      // 16-bit entries, 4 per row
            const uint32_t bulk = bytes & ~15u;   // a bulk copy moves multiples of 16 bytes
            const uint32_t tbar = smem_addr(tbars);
            volatile uint32_t *tw = reinterpret_cast<volatile uint32_t *>(tbars + 1);
            if (threadIdx.x == 0) {
                fence_proxy_async();  // the generic reads of the previous table come first
                uint32_t ok = 1;
                if (bulk) {
                    mbar_expect_s(tbar, bulk);
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_addr(tab)),
                        "l"(sdp->table_e16), "r"(bulk), "r"(tbar)
                        : "memory");
                }
                if (bytes > bulk)  // the last 8 bytes (an odd row count)
                    *reinterpret_cast<uint2 *>(tab + bulk) = __ldg(reinterpret_cast<const uint2 *>(
                        reinterpret_cast<const uint8_t *>(sdp->table_e16) + bulk));
                if (bulk) {
                    const uint32_t st = tw[1];
                    ok = wait_phase_s(tbar, st & 1u, p.err, p.wait_ns) ? 1u : 0u;
                    tw[1] = ok ? (st ^ 1u) : (st | 2u);
                }
                tw[0] = ok;
            }
            __syncthreads();  // the table has landed (thread 0 saw the barrier's phase complete)
            if (!tw[0]) aborted = true;
        }
        __syncthreads();
    };

    // One warp scans rows [row0, row0 + 32*C) of the text with subset sdp.
    auto run_rows = [&](const SubsetDev *sdp, uint32_t hot, uint64_t row0) {
        const uint32_t *gtab = sdp->table;
        const uint32_t warm = sdp->warm;
        const uint32_t warm_bytes = (FMT == FMT_U8) ? warm : (warm + 3) / 4;
        const uint32_t nW = (warm_bytes + BX - 1) / BX;
        const uint32_t L32 = p.row_bytes;
        const uint32_t nst = nW + L32 / BX;
        // Rows at or beyond full_rows (the partial last row, and rows past the
        // end of the text in the last row block) are not in the row tensor map:
        // their boxes are zero-filled or not copied. After each stage lands,
        // their lanes write their 16 bytes into the slot themselves -- the
        // partial last row its own bytes (read from global memory), the others
        // a filler of A codes whose walk is thrown away -- so that the fast
        // loop sees only letters of the alphabet.
        const bool has_oob = row0 + 32 * C > p.full_rows;
        // Stages [s_lo, s_hi) have every row of the warp inside the text (no
        // text edge): their stages need no per-chain checks.
        const uint64_t row_last = min(row0 + 32 * C, p.row_end) - 1;
        const uint64_t warm_total = (uint64_t)nW * BX;
        const uint32_t s_lo = row0 * L32 >= warm_total ? 0u : (uint32_t)(nW - row0 * L32 / BX);
        uint32_t s_hi = 0;
        {
            const int64_t spb = (FMT == FMT_U8) ? 1 : 4;
            const int64_t lim = ((int64_t)p.nsym - (int64_t)SYM) / spb - (int64_t)row_last * L32;  // max stage byte offset
            if (p.nsym >= SYM && lim >= -(int64_t)warm_total) {
                const int64_t last = (lim + (int64_t)warm_total) / BX + 1;
                s_hi = last < (int64_t)nst ? (uint32_t)last : nst;
            }
        }
        // tensor-map coordinates of stage 0 (x = byte column, dy = row delta),
        // then advanced by BX per stage without a division
        int32_t col, dy;
        {
            const uint32_t back = (uint32_t)warm_total;  // bytes before the row start
            const uint32_t rows_back = (back + L32 - 1) / L32;
            dy = -(int32_t)rows_back;
            col = (int32_t)(rows_back * L32 - back);
        }
        uint32_t bytes = 0;
#pragma unroll
        for (int j = 0; j < C; ++j)
            if (row0 + (uint64_t)j * 32 < p.full_rows) bytes += BOX;

        // lane 0 issues one 2-D box per chain group that holds a full row
        auto issue = [&]() {
            mbar_expect_s(my_bar, bytes);
#pragma unroll
            for (int j = 0; j < C; ++j)
                if (row0 + (uint64_t)j * 32 < p.full_rows)
                    tma_2d_s(my_stage + j * BOX, &rows_map, col, (int32_t)(row0 + j * 32) + dy, my_bar, xpol);
        };
        auto advance = [&]() {
            col += BX;
            if (col >= (int32_t)L32) {
                col -= (int32_t)L32;
                dy += 1;
            }
        };
        // a warp whose rows are all beyond the full rows (only the partial last
        // row) has nothing to copy: its lanes fill the slot themselves (above)
        const bool copies = bytes != 0;
        if (copies && lane == 0) issue();
        advance();
        const uint32_t rd = my_stage + lane * BX;  // this lane's row in each chain group's box

        // this warp's part of the queue of stages whose matches are emitted after the row block
        uint32_t qcount = 0;
        const uint32_t qper = p.q ? (uint32_t)(p.q_cap / ((uint64_t)gridDim.x * nwarps)) : 0u;
        EmitEntry *myq = p.q ? p.q + ((uint64_t)blockIdx.x * nwarps + warp) * qper : nullptr;
        uint32_t st[C];  // state per chain: SMEM32 row offset (| output bit), E16 id (| kFlag)
#pragma unroll
        for (int j = 0; j < C; ++j) st[j] = 0;

        for (uint32_t s = 0; s < nst; ++s) {
            if (copies) {
                if (!wait_phase_s(my_bar, parity & 1u, p.err, p.wait_ns)) {
                    aborted = true;
                    return;
                }
                parity ^= 1u;
            }
            if (has_oob) {
                const int64_t o = ((int64_t)s - (int64_t)nW) * BX;  // stage offset from the row start
                constexpr uint32_t kFill = (FMT == FMT_U8) ? 0x41414141u : 0u;  // "AAAA" (code 0)
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    const uint64_t row = row0 + (uint64_t)j * 32 + lane;
                    if (row >= p.full_rows) {
                        uint32_t v[4] = {kFill, kFill, kFill, kFill};
                        if (row == p.full_rows && row < p.row_end) {
                            // the partial last row (its box may not have been copied at all: its
                            // warm-up too); bytes outside the text stay filler
                            const int64_t b0 = (int64_t)row * L32 + o;
                            if (b0 >= 0 && b0 + 16 <= (int64_t)p.nbytes) {
                                const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p.text + b0));  // 16-byte aligned
                                v[0] = x.x;
                                v[1] = x.y;
                                v[2] = x.z;
                                v[3] = x.w;
                            } else {
                                for (int k = 0; k < 16; ++k)
                                    if (b0 + k >= 0 && b0 + k < (int64_t)p.nbytes)
                                        v[k >> 2] = (v[k >> 2] & ~(0xffu << (8 * (k & 3)))) |
                                                    ((uint32_t)__ldg(p.text + b0 + k) << (8 * (k & 3)));
                            }
                        }
                        asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(rd + j * BOX), "r"(v[0]),
                                     "r"(v[1]), "r"(v[2]), "r"(v[3])
                                     : "memory");
                    }
                }
                __syncwarp();
            }
            const bool main_stage = s >= nW;
            uint32_t u[C], acc[C], bad = 0;  // bad: bytes outside ACGT in any chain of the thread
#pragma unroll
            for (int j = 0; j < C; ++j) {
                u[j] = st[j];
                acc[j] = 0;
            }
            // The stage is read from the slot in two 8-byte halves; the slot is
            // refilled once the second half is in registers. The C chains
            // advance together, one lookup each per round, so their lookups are
            // independent and overlap. Chains off the fast path walk in-bounds
            // garbage that is discarded.
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint2 half[C];
#pragma unroll
                for (int j = 0; j < C; ++j) half[j] = lds64(rd + j * BOX + 8 * h);
                if (h == 1) {
                    __syncwarp();
                    if (s + 1 < nst) {
                        fence_proxy_async();
                        if (copies && lane == 0) issue();
                        advance();
                    }
                }
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    uint32_t cw[C];
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        const uint32_t w = e == 0 ? half[j].x : half[j].y;
                        if (FMT == FMT_U8) {
                            // ACGT -> code k in bits [SH, SH+2) of each byte (SH = 2 or 1)
                            cw[j] = LM == LEAN_SMEM32 ? ((w ^ (w << 1)) & 0x0c0c0c0cu) : ((w ^ (w >> 1)) & 0x06060606u);
                            bad |= acgt_mismatch4(w, LM == LEAN_SMEM32 ? cw[j] >> 2 : cw[j] >> 1);
                        } else {
                            cw[j] = w;
                        }
                    }
                    constexpr int PER = (FMT == FMT_U8) ? 4 : 16;
                    uint32_t prev[C];  // the previous step's entry, ORed in with the current one
#pragma unroll
                    for (int b = 0; b < PER; ++b) {
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            if (LM == LEAN_SMEM32) {
                                const uint32_t c4 =
                                    (FMT == FMT_U8) ? __byte_perm(cw[j], 0, 0x4440 + b) : packed_code<2>(cw[j], b);
                                u[j] = *reinterpret_cast<const uint32_t *>(tab + ((u[j] & ~15u) | c4));
                            } else {
                                const uint32_t c2 =
                                    (FMT == FMT_U8) ? __byte_perm(cw[j], 0, 0x4440 + b) : packed_code<1>(cw[j], b);
                                const uint32_t gi = (u[j] << 3) + c2;
                                u[j] = e16_step(u[j], sbase + gi, gi, hot, gtab);
                            }
                            if (b & 1) acc[j] |= prev[j] | u[j];
                            else prev[j] = u[j];
                        }
                    }
                }
            }
            // Common case: every chain of the warp inside the text and one vote
            // finds no lane with an output or a byte outside ACGT.
            bool slow = true, emit_only = false;
            if (s >= s_lo && s < s_hi) {
                uint32_t flags = 0;
                if (main_stage) {
#pragma unroll
                    for (int j = 0; j < C; ++j) flags |= acc[j] & FLAG;
                }
                slow = __any_sync(kFull, (flags | bad) != 0);
                // with a queue, a stage whose only reason to stop is an output
                // keeps its states and hands its matches to the emitting kernel
                emit_only = slow && p.q != nullptr && !__any_sync(kFull, bad != 0);
            }
            if (emit_only) {
                // the warp's flagged chain stages go to its own part of the queue,
                // walked again with their emission once the row block is done; a
                // part too full for them leaves the stage to the careful walk
                uint32_t total = 0;
#pragma unroll
                for (int j = 0; j < C; ++j)
                    total += __popc(__ballot_sync(kFull, (acc[j] & FLAG) != 0 && row0 + (uint64_t)j * 32 + lane < p.row_end));
                if (qcount + total <= qper) {
#pragma unroll
                    for (int j = 0; j < C; ++j) {
                        const bool f = (acc[j] & FLAG) != 0 && row0 + (uint64_t)j * 32 + lane < p.row_end;
                        const unsigned bal = __ballot_sync(kFull, f);
                        if (f) {
                            EmitEntry en;
                            en.row = (uint32_t)(row0 + (uint64_t)j * 32 + lane);
                            en.stage = s;
                            en.s = LM == LEAN_SMEM32 ? (st[j] >> 4) : (st[j] & kStateMask);
                            en.pad = 0;
                            myq[qcount + __popc(bal & ((1u << lane) - 1u))] = en;
                        }
                        qcount += __popc(bal);
                    }
#pragma unroll
                    for (int j = 0; j < C; ++j) st[j] = u[j];
                } else {
                    emit_only = false;  // the careful walk below
                }
            }
            if (!slow) {
#pragma unroll
                for (int j = 0; j < C; ++j) st[j] = u[j];
            } else if (!emit_only) {
                // chain by chain (a rolled loop over a rotation of the per-chain
                // registers, so the careful walk is inlined once): positions,
                // then a careful walk wherever a lane of the chain needs one
                const int64_t o = ((int64_t)s - (int64_t)nW) * BX;
#pragma unroll 1
                for (uint32_t jj = 0; jj < (uint32_t)C; ++jj) {
                    const uint64_t row = row0 + (uint64_t)jj * 32 + lane;
                    const int64_t b0 = (int64_t)row * L32 + o;
                    const int64_t pos0 = (FMT == FMT_U8) ? b0 : b0 * 4;
                    const bool dead = row >= p.row_end || pos0 >= nsym;
                    const bool before = !dead && pos0 + (int64_t)SYM <= 0;
                    // (the partial last row's stages were written into the slot: its stages inside the
                    // text are as good as any)
                    const bool fast = !dead && pos0 >= 0 && pos0 + (int64_t)SYM <= nsym;
                    const bool need = !dead && !before && (!fast || bad != 0 || (main_stage && (acc[0] & FLAG)));
                    uint32_t nx = u[0];
                    if (__any_sync(kFull, need)) {
                        const uint32_t s_in = LM == LEAN_SMEM32 ? (st[0] >> 4) : (st[0] & kStateMask);
                        const uint32_t sc = lean_careful<FMT, LM>(s_in, row, o, main_stage, p, sdp, tab, smap, hot, lane);
                        if (need) nx = LM == LEAN_SMEM32 ? (sc << 4) : sc;
                    }
                    nx = before ? 0u : nx;
                    // rotate: chain jj + 1 moves to index 0, chain jj's new state to index C - 1
#pragma unroll
                    for (int j = 0; j + 1 < C; ++j) {
                        u[j] = u[j + 1];
                        acc[j] = acc[j + 1];
                        st[j] = st[j + 1];
                    }
                    st[C - 1] = nx;
                }
            }
        }
        // the queued stages of this row block, walked again with their emission
        // (a lane per stage; its bytes are read again from global memory)
#pragma unroll 1
        for (uint32_t i = 0; i < qcount; i += 32) {
            EmitEntry en{0xffffffffu, 0, 0, 0};
            if (i + lane < qcount) en = myq[i + lane];
            const bool has = en.row != 0xffffffffu;
            const int64_t o = ((int64_t)en.stage - (int64_t)nW) * BX;
            lean_emit_stage<FMT, LM>(has, en.s, has ? (uint64_t)((int64_t)en.row * L32 + o) : 0, p, *sdp, tab, hot,
                                     lane);
        }
    };

    auto hot_of = [&](const SubsetDev *sdp) -> uint32_t {
        return LM == LEAN_SMEM32 ? sdp->states : min(sdp->rows_e16, p.smem_rows);
    };

    if (p.K == 1) {
        // one machine: the table is staged once and each warp takes its own
        // blocks of 32*C rows, spread over the CTAs first (a short text still
        // reaches many SMs)
        const SubsetDev *sdp = p.subs;
        const uint32_t hot = hot_of(sdp);
        stage_table(sdp, hot);
        const uint64_t blocks = (p.row_end - p.row_begin + 32 * C - 1) / (32 * C);
        for (uint64_t t = (uint64_t)warp * gridDim.x + blockIdx.x; t < blocks && !aborted;
             t += (uint64_t)gridDim.x * nwarps)
            run_rows(sdp, hot, p.row_begin + t * 32 * C);
    } else {
        // subset machines: tiles of (threads * C rows, subset), subset index
        // fastest so concurrent CTAs share text rows in L2; the table is staged
        // again when a CTA's subset changes
        int cur_k = -1;
        for (uint64_t tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
            const uint32_t k = (uint32_t)(tile % p.K);
            const SubsetDev *sdp = p.subs + k;
            const uint32_t hot = hot_of(sdp);
            if ((int)k != cur_k) {
                stage_table(sdp, hot);
                cur_k = (int)k;
            }
            if (aborted) continue;  // keeps taking part in the CTA barriers, does no work
            const uint64_t row0 = p.row_begin + (tile / p.K) * p.rows_per_tile + (uint64_t)warp * 32 * C;
            if (row0 < p.row_end) run_rows(sdp, hot, row0);
        }
    }
    // A warp that gave up inside run_rows has a text copy in flight; one that
    // stopped because a table copy was late (state word [0] = 0) has none
    // (every earlier row block waited for all of its copies).
    if (aborted && lane == 0 && reinterpret_cast<volatile uint32_t *>(tbars + 1)[0] != 0) {
        // let a copy already issued by this warp land before the CTA exits (bounded)
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait_s(my_bar, parity & 1u) && global_ns() - t0 < 100000000ull) {
        }
    }
    if (threadIdx.x == 0) {  // the same for a table copy that was late
        const uint32_t st = reinterpret_cast<volatile uint32_t *>(tbars + 1)[1];
        const uint64_t t0 = global_ns();
        while ((st & 2u) && !mbar_try_wait_s(smem_addr(tbars), st & 1u) && global_ns() - t0 < 100000000ull) {
        }
    }
}

using LeanFn = void (*)(ScanParams, CUtensorMap, CUtensorMap);

// lean shapes: (threads, chains) in {(1024, 4), (1024, 2), (768, 4), (512, 4)}
template <int FMT, int LM>
LeanFn pick_lean_shape(uint32_t threads, uint32_t C) {
    if (threads == 1024) {
        if (C == 4) return lean_kernel<FMT, LM, 4, 1024>;
        if (C == 3) return lean_kernel<FMT, LM, 3, 1024>;
        if (C == 2) return lean_kernel<FMT, LM, 2, 1024>;
    } else if (threads == 768 && C == 4) {
        return lean_kernel<FMT, LM, 4, 768>;
    } else if (threads == 512 && C == 4) {
        return lean_kernel<FMT, LM, 4, 512>;
    }
    return nullptr;
}

// defined in the scan_lean_*.cu translation units
LeanFn lean_u8_smem32(uint32_t threads, uint32_t C);
LeanFn lean_u8_e16(uint32_t threads, uint32_t C);
LeanFn lean_packed_smem32(uint32_t threads, uint32_t C);
LeanFn lean_packed_e16(uint32_t threads, uint32_t C);

}  // namespace kern
}  // namespace acgb
