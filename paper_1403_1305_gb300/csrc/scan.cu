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
#include <cub/device/device_radix_sort.cuh>

#include <cuda.h>

#include "ac_internal.h"

namespace acgb {

namespace {

constexpr int kNS = 2;           // pipeline slots per warp
constexpr uint32_t kSB = 16;     // bytes per sub-block
constexpr unsigned kFull = 0xffffffffu;

enum { FMT_U8 = 0, FMT_P2 = 1 };
enum { ALPHA_MAP = 0, ALPHA_ACGT = 1 };
enum { MODE_SMEM = 0, MODE_HYBRID = 1 };

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
    // batch mode (several texts in one arena of whole rows)
    const BatchItemDev *items;  // sorted by first row
    const BatchTileDev *tiles;  // one per tile: machine and first row
    uint32_t num_items;
    uint8_t sym_of_byte[256];
};

// ------------------------------------------------------------------ PTX helpers
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

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x, int32_t y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_1d(void *dst, const CUtensorMap *map, int32_t x, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on an mbarrier phase: false (and the error word set) after 2 s.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity, uint32_t *err) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && global_ns() - t0 > 2000000000ull) {
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

// ------------------------------------------------------------------ table lookups
template <int MODE>
__device__ __forceinline__ uint32_t lookup(const uint32_t *__restrict__ stab, const uint32_t *__restrict__ gtab,
                                           uint32_t smem_states, uint32_t sigma, uint32_t v, uint32_t c) {
    uint32_t s = v & kStateMask;
    if (MODE == MODE_SMEM) return stab[s * sigma + c];
    if (s < smem_states) return stab[s * sigma + c];
    return __ldg(gtab + (uint64_t)s * sigma + c);
}

template <int MODE>
__device__ __forceinline__ uint32_t lookup4(const uint32_t *__restrict__ stab, const uint32_t *__restrict__ gtab,
                                            uint32_t smem_states, uint32_t v, uint32_t c) {
    // sigma = 4: index = s*4 + c; the shift drops the flag bit
    uint32_t idx = (v << 2) | c;
    if (MODE == MODE_SMEM) return stab[idx];
    if ((v & kStateMask) < smem_states) return stab[idx];
    return __ldg(gtab + (((uint64_t)(v & kStateMask)) << 2) + c);
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
// stage's 32 bytes are in w0/w1 (every byte of the text inside the stage is
// there; positions before the text start reset the walk to the root). All 32
// lanes call it together; returns the state after the stage.
template <int FMT>
__device__ __noinline__ uint32_t careful_walk(uint32_t s_in, int64_t pos0, bool active, bool main_stage,
                                             const uint4 w0, const uint4 w1, const ChainText &ct,
                                             const ScanParams &p, const SubsetDev &sd, const uint32_t *stab,
                                             const uint8_t *smap, uint32_t hot, uint32_t lane) {
    constexpr uint32_t SYM = (FMT == FMT_U8) ? kStageBytes : kStageBytes * 4;
    const uint32_t w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    uint32_t sc = s_in;
    for (uint32_t i = 0; i < SYM; ++i) {
        const int64_t pos = pos0 + i;
        const bool live = active && pos >= 0 && pos < (int64_t)ct.nsym;
        bool has = false;
        if (live) {
            const uint32_t bi = (FMT == FMT_U8) ? i : (i >> 2);
            const uint32_t byte = (w[bi >> 2] >> (8 * (bi & 3))) & 0xffu;
            const uint32_t c = (FMT == FMT_U8) ? (uint32_t)smap[byte] : (byte >> (2 * (i & 3))) & 3u;
            uint32_t nv = 0;
            if (c < p.sigma) nv = lookup<MODE_HYBRID>(stab, sd.table, hot, p.sigma, sc, c);
            sc = nv & kStateMask;
            has = main_stage && (nv & kFlag);
        } else if (pos < 0) {
            sc = 0;
        }
        emit_warp(has, sc, ct.vbase + (uint64_t)(pos < 0 ? 0 : pos), ct.cbase, sd, p, lane);
    }
    return sc;
}

// ------------------------------------------------------------------ the kernel
// Shared memory per warp and pipeline slot: C boxes of 32 rows x 32 bytes
// (one per chain group, written by one 2-D TMA each) and one 32-byte slot
// for the ragged last row (written by a 1-D TMA), padded to 128 bytes.
__host__ __device__ constexpr uint32_t slot_bytes_for(uint32_t C) { return C * 1024u + 128u; }

// The chain's text: in single-text mode the row index is the text row; in
// batch mode the row's text is found by binary search over the items.
template <bool BATCH>
__device__ __forceinline__ bool chain_text(uint64_t row, const ScanParams &p, ChainText &ct) {
    if (!BATCH) {
        ct.row_in_text = row;
        ct.nsym = p.nsym;
        ct.vbase = 0;
        ct.cbase = 0;
        return row < p.num_rows;
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

template <int FMT, int ALPHA, int MODE, int C, bool BATCH>
__global__ void __launch_bounds__(512, 1)
    scan_kernel(const __grid_constant__ ScanParams p, const __grid_constant__ CUtensorMap rows_map,
                const __grid_constant__ CUtensorMap tail_map) {
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr uint32_t BX = kStageBytes;
    constexpr uint32_t SYM_PER_STAGE = (FMT == FMT_U8) ? BX : BX * 4;
    constexpr uint32_t SLOT = slot_bytes_for(C);

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
            tile_row0 = (tile / p.K) * p.rows_per_tile;
        }
        const SubsetDev sd = p.subs[k];
        const uint32_t hot = min(sd.states, p.smem_rows);
        if ((int)k != cur_k) {
            __syncthreads();  // every warp is done with the previous table
            const uint32_t words = hot * sigma;
            const uint4 *src4 = reinterpret_cast<const uint4 *>(sd.table);
            uint4 *dst4 = reinterpret_cast<uint4 *>(stab);
            for (uint32_t i = threadIdx.x; i < words / 4; i += blockDim.x) dst4[i] = __ldg(src4 + i);
            for (uint32_t i = (words & ~3u) + threadIdx.x; i < words; i += blockDim.x) stab[i] = __ldg(sd.table + i);
            __syncthreads();
            cur_k = (int)k;
        }
        if (aborted) continue;  // keeps taking part in the CTA barriers above, does no work

        const uint32_t warm_bytes = (FMT == FMT_U8) ? sd.warm : (sd.warm + 3) / 4;
        const uint32_t nW = (warm_bytes + BX - 1) / BX;
        const uint32_t nst = nW + p.row_bytes / BX;
        const uint64_t row0 = tile_row0 + (uint64_t)warp * 32 * C;
        if (row0 >= p.num_rows) continue;
        const bool tail_in_warp = !BATCH && p.tail_bytes && p.full_rows >= row0 && p.full_rows < row0 + 32 * C;

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
                if (row0 + (uint64_t)j * 32 < p.num_rows) bytes += 1024;
            const bool tail_now = tail_in_warp && o >= 0;
            if (tail_now) bytes += BX;
            mbar_arrive_expect_tx(bar, bytes);
#pragma unroll
            for (int j = 0; j < C; ++j)
                if (row0 + (uint64_t)j * 32 < p.num_rows)
                    tma_load_2d(base + j * 1024, &rows_map, col, (int32_t)((int64_t)(row0 + j * 32) + dy), bar);
            if (tail_now) tma_load_1d(base + C * 1024, &tail_map, (int32_t)o, bar);
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
            if (!wait_phase(my_bars + slot, (parity >> slot) & 1u, p.err)) {
                aborted = true;
                break;
            }
            parity ^= 1u << slot;
            const int64_t o = (int64_t)s * BX - (int64_t)nW * BX;
            const bool main_stage = o >= 0;
            // this stage's 32 bytes of every chain into registers, then refill the slot
            uint4 data[C][2];
            const uint8_t *base = my_stage + slot * SLOT;
            const uint32_t swz = (lane >> 2) & 1u;  // lanes l and l+4 read different 16-byte halves first
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const bool tail_row = tail_in_warp && main_stage && row[j] == p.full_rows;
                const uint4 *b4 = reinterpret_cast<const uint4 *>(tail_row ? base + C * 1024 : base + j * 1024 + lane * BX);
                const uint4 t0 = b4[swz], t1 = b4[swz ^ 1u];
                data[j][0] = swz ? t1 : t0;
                data[j][1] = swz ? t0 : t1;
            }
            __syncwarp();
            if (s + kNS < nst) {
                fence_proxy_async();
                if (lane == 0) issue(s + kNS);
            }

            int64_t pos0[C];
            bool fast[C], dead[C], before[C];
            uint32_t v[C], acc[C], bad[C], s_in[C];
#pragma unroll
            for (int j = 0; j < C; ++j) {
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
            // The C chains advance together, one symbol each per round, so their
            // lookups are independent and overlap. Chains off the fast path walk
            // in-bounds garbage that is discarded.
            if (FMT == FMT_U8 && ALPHA == ALPHA_ACGT) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
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
                            v[j] = lookup4<MODE>(stab, sd.table, hot, v[j], (cw[j] >> (8 * b)) & 3u);
                            acc[j] |= v[j];
                        }
                    }
                }
            } else if (FMT == FMT_U8) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            const uint32_t c = smap[(word_of(data[j][e >> 2], e & 3) >> (8 * b)) & 0xffu];
                            const uint32_t nv = lookup<MODE>(stab, sd.table, hot, sigma, v[j], c < sigma ? c : 0u);
                            v[j] = c < sigma ? nv : 0u;
                            acc[j] |= v[j];
                        }
                    }
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
#pragma unroll
                    for (int b = 0; b < 16; ++b) {
#pragma unroll
                        for (int j = 0; j < C; ++j) {
                            v[j] = lookup4<MODE>(stab, sd.table, hot, v[j], (word_of(data[j][e >> 2], e & 3) >> (2 * b)) & 3u);
                            acc[j] |= v[j];
                        }
                    }
                }
            }
            bool need[C];
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if (fast[j]) st8[j] = v[j] & kStateMask;
                else if (before[j]) st8[j] = 0;
                need[j] = !dead[j] && !before[j] && (!fast[j] || bad[j] != 0 || (main_stage && (acc[j] & kFlag)));
            }
#pragma unroll
            for (int j = 0; j < C; ++j) {
                if (__any_sync(kFull, need[j])) {
                    const uint32_t sc = careful_walk<FMT>(s_in[j], pos0[j], active[j], main_stage, data[j][0],
                                                          data[j][1], ct[j], p, sd, stab, smap, hot, lane);
                    if (!dead[j]) st8[j] = sc;
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

// ------------------------------------------------------------------ small kernels
__global__ void fill_u64_kernel(unsigned long long *p, uint64_t count, unsigned long long value) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = value;
}

__global__ void keys_to_matches_kernel(const unsigned long long *__restrict__ keys, const unsigned long long *num,
                                       uint64_t cap, uint32_t shift, ac_match *__restrict__ out,
                                       unsigned long long *num_out, const uint32_t *err) {
    const unsigned long long M = *num;
    const uint64_t m = M < cap ? M : cap;
    const unsigned long long mask = (1ull << shift) - 1ull;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long k = keys[i];
        ac_match r;
        r.pos = (uint32_t)(k >> shift);
        r.pattern_id = (uint32_t)(k & mask);
        out[i] = r;
    }
    if (num_out && blockIdx.x == 0 && threadIdx.x == 0) *num_out = (err && *err) ? ~0ull : M;
}

// keys[i] for i in [*num, cap) := all ones (sorts after every real key)
__global__ void pad_keys_kernel(unsigned long long *keys, const unsigned long long *num, uint64_t cap) {
    const unsigned long long M = *num;
    for (uint64_t i = M + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap; i += (uint64_t)gridDim.x * blockDim.x)
        keys[i] = ~0ull;
}

// *num := UINT64_MAX when a device-side wait ran out
__global__ void mark_error_kernel(unsigned long long *num, const uint32_t *err) {
    if (*err) *num = ~0ull;
}

// ------------------------------------------------------------------ dispatch
using KernelFn = void (*)(ScanParams, CUtensorMap, CUtensorMap);

template <int FMT, int ALPHA, int MODE, bool BATCH>
KernelFn pick_c(uint32_t C) {
    switch (C) {
        case 1: return scan_kernel<FMT, ALPHA, MODE, 1, BATCH>;
        case 2: return scan_kernel<FMT, ALPHA, MODE, 2, BATCH>;
        default: return scan_kernel<FMT, ALPHA, MODE, 4, BATCH>;
    }
}

template <bool BATCH>
KernelFn pick_mode(int fmt, bool acgt, bool hybrid, uint32_t C) {
    if (fmt == AC_PACKED2)
        return hybrid ? pick_c<FMT_P2, ALPHA_MAP, MODE_HYBRID, BATCH>(C)
                      : pick_c<FMT_P2, ALPHA_MAP, MODE_SMEM, BATCH>(C);
    if (acgt)
        return hybrid ? pick_c<FMT_U8, ALPHA_ACGT, MODE_HYBRID, BATCH>(C)
                      : pick_c<FMT_U8, ALPHA_ACGT, MODE_SMEM, BATCH>(C);
    return hybrid ? pick_c<FMT_U8, ALPHA_MAP, MODE_HYBRID, BATCH>(C) : pick_c<FMT_U8, ALPHA_MAP, MODE_SMEM, BATCH>(C);
}

KernelFn pick_kernel(int fmt, bool acgt, bool hybrid, uint32_t C, bool batch) {
    return batch ? pick_mode<true>(fmt, acgt, hybrid, C) : pick_mode<false>(fmt, acgt, hybrid, C);
}

uint32_t bits_for(uint64_t x) {  // bits needed to hold values 0..x
    uint32_t b = 1;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(f);
    });
    return fn;
}

// rows x row_bytes bytes at base, boxes of 32 bytes x 32 rows
int encode_rows_map(CUtensorMap *m, const uint8_t *base, uint64_t row_bytes, uint64_t rows) {
    EncodeTiled enc = encoder();
    if (!enc) return set_error(AC_ECUDA, "scan: cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[2] = {row_bytes, rows};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {kStageBytes, 32};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? AC_OK : set_error(AC_ECUDA, "scan: encoding the row tensor map failed (%d)", (int)r);
}

// bytes bytes at base, boxes of 32 bytes
int encode_tail_map(CUtensorMap *m, const uint8_t *base, uint64_t bytes) {
    EncodeTiled enc = encoder();
    if (!enc) return set_error(AC_ECUDA, "scan: cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[1] = {bytes};
    cuuint64_t strides[1] = {0};
    cuuint32_t box[1] = {kStageBytes};
    cuuint32_t es[1] = {1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, (void *)base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? AC_OK : set_error(AC_ECUDA, "scan: encoding the tail tensor map failed (%d)", (int)r);
}

}  // namespace

int scan_smem_limit(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 0;
    return v;
}

uint32_t scan_stage_bytes_per_cta(const ac_scan_config &cfg) {
    const uint32_t warps = cfg.threads / 32;
    return 256 + 128 + 128 + warps * kNS * slot_bytes_for(cfg.chains) + warps * kNS * 8;
}

void default_config(const ac_automaton *a, uint64_t n, int fmt, ac_scan_config *cfg) {
    ac_scan_config c = a->cfg;
    if (!c.threads) c.threads = 512;
    if (!c.chains) c.chains = 2;
    if (!c.row_len) {
        // one chain per row, all chains of the GPU busy once, rows at least
        // 8x the warm-up and 256 symbols long
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, a->device < 0 ? 0 : a->device);
        uint64_t chains = (uint64_t)sms * c.threads * c.chains;
        uint64_t want = (n + chains - 1) / (chains ? chains : 1);
        uint64_t lo = std::max<uint64_t>(256, 8ull * a->max_len);
        uint64_t L = std::max<uint64_t>(want, lo);
        if (L > (1u << 20)) L = 1u << 20;
        c.row_len = (uint32_t)L;
    }
    *cfg = c;
}

int key_shift_for(const ac_automaton *a) { return (int)bits_for(a->P ? a->P - 1 : 0); }

int plan_smem(int device, const ac_scan_config &cfg, uint32_t sigma, int placement, uint32_t smem_cap,
              uint32_t max_states, uint32_t *rows_used, bool *hybrid, size_t *smem_bytes, uint32_t *table_words) {
    // shared memory: table prefix (rounded to 128 bytes) + map + staging + barriers
    const int limit = scan_smem_limit(device);
    const uint32_t staging = scan_stage_bytes_per_cta(cfg);
    if ((int)staging + 1024 > limit) return set_error(AC_EINVAL, "scan: staging does not fit in shared memory");
    uint64_t avail = (uint64_t)limit - staging - 128;
    if (smem_cap && smem_cap < avail) avail = smem_cap;
    uint32_t rows_fit = (uint32_t)(avail / (4ull * sigma));
    if (placement == AC_PLACE_GLOBAL) rows_fit = 0;
    *hybrid = max_states > rows_fit;
    if (placement == AC_PLACE_SMEM && *hybrid)
        return set_error(AC_ERANGE, "scan: table of %u states does not fit in shared memory (%u rows)", max_states,
                         rows_fit);
    *rows_used = std::min(max_states, rows_fit);
    *table_words = (*rows_used * sigma + 3) & ~3u;
    *smem_bytes = (((size_t)*table_words * 4 + 127) & ~(size_t)127) + staging;
    if (*smem_bytes > (size_t)limit) return set_error(AC_EINVAL, "scan: shared memory plan exceeds the limit");
    return AC_OK;
}

int launch_scan_batch(const BatchLaunch &b, const ScanOut &o, cudaStream_t stream) {
    const ac_scan_config &cfg = b.cfg;
    if (cfg.threads < 32 || cfg.threads > 512 || cfg.threads % 32 || (cfg.chains != 1 && cfg.chains != 2 &&
                                                                        cfg.chains != 4))
        return set_error(AC_EINVAL, "batch: bad threads/chains");
    if (b.num_tiles == 0) return AC_OK;
    if (b.row_bytes % kStageBytes || ((uintptr_t)b.arena & 15))
        return set_error(AC_EINVAL, "batch: arena rows must be 32-byte multiples at a 16-byte aligned address");
    ScanParams p{};
    p.text = b.arena;
    p.nbytes = b.rows * b.row_bytes;
    p.nsym = 0;
    p.full_rows = b.rows;
    p.num_rows = b.rows;
    p.num_tiles = b.num_tiles;
    p.row_bytes = b.row_bytes;
    p.rows_per_tile = cfg.threads * cfg.chains;
    p.K = 1;
    p.sigma = b.sigma;
    p.subs = b.machines;
    p.keys = o.keys;
    p.cap = o.cap;
    p.num = o.num;
    p.counts = o.counts;
    p.err = o.err;
    p.key_shift = b.key_shift;
    p.tail_bytes = 0;
    p.items = b.items;
    p.tiles = b.tiles;
    p.num_items = b.num_items;
    memcpy(p.sym_of_byte, b.sym_of_byte, 256);
    if (b.rows >= (1ull << 31)) return set_error(AC_ERANGE, "batch: arena too large for one launch");
    CUtensorMap rows_map, tail_map;
    memset(&tail_map, 0, sizeof(tail_map));
    int rc = encode_rows_map(&rows_map, b.arena, b.row_bytes, b.rows);
    if (rc) return rc;
    uint32_t rows_used = 0;
    bool hybrid = false;
    size_t smem = 0;
    rc = plan_smem(b.device, cfg, b.sigma, b.placement, b.smem_cap_bytes, b.max_states, &rows_used, &hybrid, &smem,
                   &p.table_words);
    if (rc) return rc;
    p.smem_rows = rows_used;
    KernelFn fn = pick_kernel(b.fmt, b.fmt == AC_U8 && b.acgt, hybrid, cfg.chains, true);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(AC_ECUDA, "batch: %s", cudaGetErrorString(e));
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b.device);
    uint64_t grid = cfg.ctas ? cfg.ctas : (uint64_t)sms;
    if (grid > b.num_tiles) grid = b.num_tiles;
    fn<<<(unsigned)grid, cfg.threads, smem, stream>>>(p, rows_map, tail_map);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(AC_ECUDA, "batch launch: %s", cudaGetErrorString(e));
    return AC_OK;
}

int launch_scan(const ac_automaton *a, const ScanText &t, const ScanOut &o, const ac_scan_config &cfg_in,
                cudaStream_t stream) {
    ac_scan_config cfg = cfg_in;
    if (cfg.threads < 32 || cfg.threads > 512 || cfg.threads % 32)
        return set_error(AC_EINVAL, "scan: threads per CTA must be a multiple of 32 in [32, 512]");
    if (cfg.chains != 1 && cfg.chains != 2 && cfg.chains != 4)
        return set_error(AC_EINVAL, "scan: chains per thread must be 1, 2 or 4");
    const uint64_t nbytes = (t.fmt == AC_U8) ? t.n : (t.n + 3) / 4;
    if (nbytes == 0) return AC_OK;
    const uint64_t readable = std::max(nbytes, t.readable);
    if (readable < kStageBytes) return set_error(AC_EINVAL, "scan: text buffer shorter than one stage");
    if ((uintptr_t)t.d_text & 15) return set_error(AC_EINVAL, "scan: text must be 16-byte aligned");
    const uint32_t sym_per_byte = (t.fmt == AC_U8) ? 1 : 4;
    uint64_t rb = ((uint64_t)cfg.row_len + sym_per_byte - 1) / sym_per_byte;
    rb = (rb + kStageBytes - 1) / kStageBytes * kStageBytes;
    if (rb > (1u << 24)) rb = 1u << 24;
    const uint64_t rmax = readable / kStageBytes * kStageBytes;
    if (rb > rmax) rb = rmax;
    if (rb == 0) rb = kStageBytes;

    ScanParams p{};
    p.text = t.d_text;
    p.nbytes = nbytes;
    p.nsym = t.n;
    p.row_bytes = (uint32_t)rb;
    p.full_rows = readable / rb;
    const uint64_t covered = p.full_rows * rb;
    p.tail_bytes = nbytes > covered ? (uint32_t)(nbytes - covered) : 0u;
    p.num_rows = p.full_rows + (p.tail_bytes ? 1 : 0);
    p.rows_per_tile = cfg.threads * cfg.chains;
    p.K = a->K;
    p.sigma = a->sigma;
    p.subs = a->d_desc;
    p.keys = o.keys;
    p.cap = o.cap;
    p.num = o.num;
    p.counts = o.counts;
    p.err = o.err;
    p.key_shift = (uint32_t)key_shift_for(a);
    memcpy(p.sym_of_byte, a->sym_of_byte, 256);
    const uint64_t row_blocks = (p.num_rows + p.rows_per_tile - 1) / p.rows_per_tile;
    p.num_tiles = row_blocks * a->K;
    if (p.full_rows >= (1ull << 31) || p.num_rows * rb >= (1ull << 40))
        return set_error(AC_ERANGE, "scan: text too long for the row tensor map");

    CUtensorMap rows_map, tail_map;
    memset(&rows_map, 0, sizeof(rows_map));
    memset(&tail_map, 0, sizeof(tail_map));
    int rc = encode_rows_map(&rows_map, t.d_text, rb, p.full_rows);
    if (rc) return rc;
    if (p.tail_bytes) {
        rc = encode_tail_map(&tail_map, t.d_text + covered, p.tail_bytes);
        if (rc) return rc;
    }

    uint32_t max_states = 0;
    for (auto &d : a->h_desc) max_states = std::max(max_states, d.states);
    uint32_t rows_used = 0;
    bool hybrid = false;
    size_t smem = 0;
    rc = plan_smem(a->device, cfg, a->sigma, a->placement, a->smem_cap_bytes, max_states, &rows_used, &hybrid, &smem,
                   &p.table_words);
    if (rc) return rc;
    p.smem_rows = rows_used;

    const bool acgt = t.fmt == AC_U8 && a->dna_acgt;
    KernelFn fn = pick_kernel(t.fmt, acgt, hybrid, cfg.chains, false);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(AC_ECUDA, "scan: %s", cudaGetErrorString(e));
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, a->device);
    uint64_t grid = cfg.ctas ? cfg.ctas : (uint64_t)sms;
    if (grid > p.num_tiles) grid = p.num_tiles;
    fn<<<(unsigned)grid, cfg.threads, smem, stream>>>(p, rows_map, tail_map);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(AC_ECUDA, "scan launch: %s", cudaGetErrorString(e));
    return AC_OK;
}

int launch_fill_u64(unsigned long long *ptr, uint64_t count, unsigned long long value, cudaStream_t stream) {
    if (!count) return AC_OK;
    uint64_t blocks = (count + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    fill_u64_kernel<<<(unsigned)blocks, 256, 0, stream>>>(ptr, count, value);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AC_OK : set_error(AC_ECUDA, "fill: %s", cudaGetErrorString(e));
}

int launch_keys_to_matches(const unsigned long long *keys, const unsigned long long *num, uint64_t cap,
                           uint32_t shift, ac_match *out, unsigned long long *num_out, const uint32_t *err,
                           cudaStream_t stream) {
    uint64_t blocks = (cap + 255) / 256;
    if (blocks == 0) blocks = 1;
    if (blocks > 2048) blocks = 2048;
    keys_to_matches_kernel<<<(unsigned)blocks, 256, 0, stream>>>(keys, num, cap, shift, out, num_out, err);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AC_OK : set_error(AC_ECUDA, "convert: %s", cudaGetErrorString(e));
}

int launch_pad_keys(unsigned long long *keys, const unsigned long long *num, uint64_t cap, cudaStream_t stream) {
    uint64_t blocks = (cap + 255) / 256;
    if (blocks == 0) return AC_OK;
    if (blocks > 2048) blocks = 2048;
    pad_keys_kernel<<<(unsigned)blocks, 256, 0, stream>>>(keys, num, cap);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AC_OK : set_error(AC_ECUDA, "pad: %s", cudaGetErrorString(e));
}

int launch_mark_error(unsigned long long *num, const uint32_t *err, cudaStream_t stream) {
    mark_error_kernel<<<1, 1, 0, stream>>>(num, err);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AC_OK : set_error(AC_ECUDA, "mark: %s", cudaGetErrorString(e));
}

int sort_keys(unsigned long long *keys, unsigned long long *keys_alt, uint64_t count, int end_bit, void *temp,
              size_t *temp_bytes, cudaStream_t stream, unsigned long long **sorted) {
    if (count > 0x7fffffffull) return set_error(AC_ERANGE, "sort: too many matches");
    cub::DoubleBuffer<unsigned long long> db(keys, keys_alt);
    cudaError_t e = cub::DeviceRadixSort::SortKeys(temp, *temp_bytes, db, (int)count, 0, end_bit, stream);
    if (e != cudaSuccess) return set_error(AC_ECUDA, "sort: %s", cudaGetErrorString(e));
    if (sorted) *sorted = db.Current();
    return AC_OK;
}

}  // namespace acgb
