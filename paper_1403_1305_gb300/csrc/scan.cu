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

#include "ac_internal.h"

namespace acgb {

namespace {

constexpr int kNS = 2;           // pipeline slots per warp
constexpr uint32_t kSB = 16;     // bytes per sub-block
constexpr unsigned kFull = 0xffffffffu;

enum { FMT_U8 = 0, FMT_P2 = 1 };
enum { ALPHA_MAP = 0, ALPHA_ACGT = 1 };
enum { MODE_SMEM = 0, MODE_HYBRID = 1 };

struct ScanParams {
    const uint8_t *text;
    uint64_t nbytes;        // bytes of text
    uint64_t nbytes_al;     // nbytes rounded down to 16 (bulk copies stop there)
    uint64_t nsym;          // symbols
    uint64_t num_rows;
    uint64_t num_tiles;
    uint32_t row_bytes;     // multiple of kStageBytes
    uint32_t rows_per_tile; // warps * 32 * C
    uint32_t K;
    uint32_t sigma;
    uint32_t smem_rows;     // table rows that fit in shared memory
    uint32_t table_words;   // words reserved for the table in shared memory
    uint32_t key_shift;     // key = pos << key_shift | id
    const SubsetDev *subs;
    unsigned long long *keys;
    uint64_t cap;
    unsigned long long *num;
    unsigned long long *counts;
    uint32_t *err;
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

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
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
__device__ __forceinline__ void emit_warp(bool has, uint32_t sid, uint64_t pos, const SubsetDev &sd,
                                          const ScanParams &p, uint32_t lane) {
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
        if (p.counts) atomicAdd(p.counts + id, 1ull);
    }
}

// ------------------------------------------------------------------ the kernel
template <int FMT, int ALPHA, int MODE, int C>
__global__ void __launch_bounds__(512, 1) scan_kernel(const __grid_constant__ ScanParams p) {
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr uint32_t BX = kStageBytes;
    constexpr uint32_t SYM_PER_SB = (FMT == FMT_U8) ? kSB : kSB * 4;

    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t *stab = reinterpret_cast<uint32_t *>(smem);
    uint8_t *smap = smem + (size_t)p.table_words * 4;
    uint8_t *stage = smap + 256;
    const uint32_t warp_stage_bytes = kNS * C * 32 * BX;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage + (size_t)nwarps * warp_stage_bytes);
    uint8_t *my_stage = stage + (size_t)warp * warp_stage_bytes;
    uint64_t *my_bars = bars + warp * kNS;

    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) smap[i] = p.sym_of_byte[i];
    if (threadIdx.x == 0) {
        for (uint32_t i = 0; i < nwarps * kNS; ++i) mbar_init(bars + i, 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t parity = 0;  // bit i = expected parity of slot i
    bool aborted = false;
    int cur_k = -1;
    const uint32_t sigma = p.sigma;

    for (uint64_t tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
        const uint32_t k = (uint32_t)(tile % p.K);
        const uint64_t rb = tile / p.K;
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
        // warm-up stages for this subset
        const uint32_t warm_bytes = (FMT == FMT_U8) ? sd.warm : (sd.warm + 3) / 4;
        const uint32_t nW = (warm_bytes + BX - 1) / BX;
        const uint32_t nst = nW + p.row_bytes / BX;

        // this warp's chains
        const uint64_t row0 = rb * p.rows_per_tile + (uint64_t)warp * 32 * C;
        int64_t x0[C];
        bool active[C];
        uint32_t st8[C];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            uint64_t row = row0 + (uint64_t)j * 32 + lane;
            active[j] = row < p.num_rows;
            x0[j] = (int64_t)(row * p.row_bytes) - (int64_t)nW * BX;
            st8[j] = 0;
        }

        auto issue = [&](uint32_t s) {
            const uint32_t slot = s % kNS;
            uint8_t *buf = my_stage + slot * (C * 32 * BX);
            uint32_t bytes[C], total = 0;
            int64_t lo[C];
#pragma unroll
            for (int j = 0; j < C; ++j) {
                int64_t x = x0[j] + (int64_t)s * BX;
                int64_t l = x > 0 ? x : 0;
                int64_t h = x + BX < (int64_t)p.nbytes_al ? x + BX : (int64_t)p.nbytes_al;
                bytes[j] = (active[j] && h > l) ? (uint32_t)(h - l) : 0u;
                lo[j] = l;
                total += bytes[j];
            }
            mbar_arrive_expect_tx(my_bars + slot, total);
#pragma unroll
            for (int j = 0; j < C; ++j)
                if (bytes[j])
                    bulk_copy_g2s(buf + (j * 32 + lane) * BX + (lo[j] - (x0[j] + (int64_t)s * BX)), p.text + lo[j],
                                  bytes[j], my_bars + slot);
        };

        if (aborted) continue;  // keeps taking part in the CTA barriers above, does no work
        for (uint32_t s = 0; s < (uint32_t)kNS && s < nst; ++s) issue(s);

        for (uint32_t s = 0; s < nst; ++s) {
            const uint32_t slot = s % kNS;
            if (!wait_phase(my_bars + slot, (parity >> slot) & 1u, p.err)) {
                aborted = true;
                break;
            }
            parity ^= 1u << slot;
            // read this stage's bytes into registers, then refill the slot
            uint4 data[C][BX / 16];
            const uint8_t *buf = my_stage + slot * (C * 32 * BX);
            const uint32_t swz = (lane >> 2) & 1u;  // avoids 2-way bank conflicts between lanes l and l+4
#pragma unroll
            for (int j = 0; j < C; ++j) {
                const uint4 *b4 = reinterpret_cast<const uint4 *>(buf + (j * 32 + lane) * BX);
#pragma unroll
                for (uint32_t q = 0; q < BX / 16; ++q) {
                    uint32_t qq = q ^ swz;
                    uint4 t = b4[qq];
                    if (qq == 0) data[j][0] = t; else data[j][1] = t;
                }
            }
            __syncwarp();
            fence_proxy_async();
            if (s + kNS < nst) issue(s + kNS);

            const bool main_stage = s >= nW;
#pragma unroll
            for (int j = 0; j < C; ++j) {
#pragma unroll
                for (uint32_t q = 0; q < BX / 16; ++q) {
                    const int64_t b0 = x0[j] + (int64_t)s * BX + (int64_t)q * kSB;  // byte offset of sub-block
                    const int64_t pos0 = (FMT == FMT_U8) ? b0 : b0 * 4;           // symbol position of its start
                    const bool dead = !active[j] || pos0 >= (int64_t)p.nsym;
                    const bool before = !dead && pos0 + (int64_t)SYM_PER_SB <= 0;
                    const bool fast = !dead && !before && b0 >= 0 && b0 + (int64_t)kSB <= (int64_t)p.nbytes_al &&
                                      pos0 + (int64_t)SYM_PER_SB <= (int64_t)p.nsym;
                    const uint32_t s_in = st8[j];
                    uint32_t v = s_in, acc = 0, bad = 0;
                    const uint4 w4 = data[j][q];
                    const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
                    if (fast) {
                        if (FMT == FMT_U8 && ALPHA == ALPHA_ACGT) {
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                uint32_t cw = acgt_codes4(w[e]);
                                bad |= acgt_mismatch4(w[e], cw);
#pragma unroll
                                for (int b = 0; b < 4; ++b) {
                                    v = lookup4<MODE>(stab, sd.table, hot, v, (cw >> (8 * b)) & 3u);
                                    acc |= v;
                                }
                            }
                        } else if (FMT == FMT_U8) {
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
#pragma unroll
                                for (int b = 0; b < 4; ++b) {
                                    uint32_t c = smap[(w[e] >> (8 * b)) & 0xffu];
                                    uint32_t cc = c < sigma ? c : 0u;
                                    uint32_t nv = lookup<MODE>(stab, sd.table, hot, sigma, v, cc);
                                    v = c < sigma ? nv : 0u;
                                    acc |= v;
                                }
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
#pragma unroll
                                for (int b = 0; b < 16; ++b) {
                                    v = lookup4<MODE>(stab, sd.table, hot, v, (w[e] >> (2 * b)) & 3u);
                                    acc |= v;
                                }
                            }
                        }
                        st8[j] = v & kStateMask;
                    } else if (before) {
                        st8[j] = 0;
                    }
                    const bool need = !dead && !before && (!fast || bad != 0 || (main_stage && (acc & kFlag)));
                    if (__any_sync(kFull, need)) {
                        // careful walk of this sub-block, all lanes together
                        uint32_t sc = s_in;
                        for (uint32_t i = 0; i < SYM_PER_SB; ++i) {
                            const int64_t pos = pos0 + i;
                            const bool live = active[j] && pos >= 0 && pos < (int64_t)p.nsym;
                            bool has = false;
                            if (live) {
                                const int64_t boff = (FMT == FMT_U8) ? pos : (pos >> 2);
                                uint32_t byte;
                                if (boff < (int64_t)p.nbytes_al) {
                                    const uint32_t bi = (uint32_t)(boff - b0);
                                    byte = (w[bi >> 2] >> (8 * (bi & 3))) & 0xffu;
                                } else {
                                    byte = p.text[boff];
                                }
                                uint32_t c;
                                if (FMT == FMT_U8) {
                                    c = smap[byte];
                                } else {
                                    c = (byte >> (2 * (pos & 3))) & 3u;
                                }
                                uint32_t nv = 0;
                                if (c < sigma) nv = lookup<MODE_HYBRID>(stab, sd.table, hot, sigma, sc, c);
                                sc = nv & kStateMask;
                                has = main_stage && (nv & kFlag);
                            } else if (pos < 0) {
                                sc = 0;
                            }
                            emit_warp(has, sc, (uint64_t)(pos < 0 ? 0 : pos), sd, p, lane);
                        }
                        if (!dead) st8[j] = sc;
                    }
                }
            }
        }
    }
    if (aborted) {
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
using KernelFn = void (*)(ScanParams);

template <int FMT, int ALPHA, int MODE>
KernelFn pick_c(uint32_t C) {
    switch (C) {
        case 1: return scan_kernel<FMT, ALPHA, MODE, 1>;
        case 2: return scan_kernel<FMT, ALPHA, MODE, 2>;
        default: return scan_kernel<FMT, ALPHA, MODE, 4>;
    }
}

KernelFn pick_kernel(int fmt, bool acgt, bool hybrid, uint32_t C) {
    if (fmt == AC_PACKED2)
        return hybrid ? pick_c<FMT_P2, ALPHA_MAP, MODE_HYBRID>(C) : pick_c<FMT_P2, ALPHA_MAP, MODE_SMEM>(C);
    if (acgt)
        return hybrid ? pick_c<FMT_U8, ALPHA_ACGT, MODE_HYBRID>(C) : pick_c<FMT_U8, ALPHA_ACGT, MODE_SMEM>(C);
    return hybrid ? pick_c<FMT_U8, ALPHA_MAP, MODE_HYBRID>(C) : pick_c<FMT_U8, ALPHA_MAP, MODE_SMEM>(C);
}

uint32_t bits_for(uint64_t x) {  // bits needed to hold values 0..x
    uint32_t b = 1;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

}  // namespace

int scan_smem_limit(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 0;
    return v;
}

uint32_t scan_stage_bytes_per_cta(const ac_scan_config &cfg) {
    return (cfg.threads / 32) * kNS * cfg.chains * 32 * kStageBytes + (cfg.threads / 32) * kNS * 8 + 256;
}

void default_config(const ac_automaton *a, uint64_t n, int fmt, ac_scan_config *cfg) {
    ac_scan_config c = a->cfg;
    if (!c.threads) c.threads = 256;
    if (!c.chains) c.chains = 4;
    if (!c.row_len) {
        // enough rows for ~2 tiles per SM, but at least 8x the warm-up and 256 symbols
        int sms = 148;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, a->device < 0 ? 0 : a->device);
        uint64_t chains = (uint64_t)sms * c.threads * c.chains;
        uint64_t want = n / (chains ? chains : 1);
        uint64_t lo = std::max<uint64_t>(256, 8ull * a->max_len);
        uint64_t L = std::max<uint64_t>(want, lo);
        if (L > (1u << 20)) L = 1u << 20;
        c.row_len = (uint32_t)L;
    }
    *cfg = c;
}

int key_shift_for(const ac_automaton *a) { return (int)bits_for(a->P ? a->P - 1 : 0); }

int launch_scan(const ac_automaton *a, const ScanText &t, const ScanOut &o, const ac_scan_config &cfg_in,
                cudaStream_t stream) {
    ac_scan_config cfg = cfg_in;
    if (cfg.threads < 32 || cfg.threads > 512 || cfg.threads % 32)
        return set_error(AC_EINVAL, "scan: threads per CTA must be a multiple of 32 in [32, 512]");
    if (cfg.chains != 1 && cfg.chains != 2 && cfg.chains != 4)
        return set_error(AC_EINVAL, "scan: chains per thread must be 1, 2 or 4");
    const uint64_t nbytes = (t.fmt == AC_U8) ? t.n : (t.n + 3) / 4;
    if (nbytes == 0) return AC_OK;
    const uint32_t sym_per_byte = (t.fmt == AC_U8) ? 1 : 4;
    uint64_t rb = ((uint64_t)cfg.row_len + sym_per_byte - 1) / sym_per_byte;
    rb = (rb + kStageBytes - 1) / kStageBytes * kStageBytes;
    if (rb == 0) rb = kStageBytes;
    if (rb > (1u << 24)) rb = 1u << 24;

    ScanParams p{};
    p.text = t.d_text;
    p.nbytes = nbytes;
    p.nbytes_al = nbytes & ~15ull;
    p.nsym = t.n;
    p.row_bytes = (uint32_t)rb;
    p.num_rows = (nbytes + rb - 1) / rb;
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

    // shared memory: table prefix + map + staging + barriers
    const int limit = scan_smem_limit(a->device);
    const uint32_t staging = scan_stage_bytes_per_cta(cfg);
    if ((int)staging + 1024 > limit) return set_error(AC_EINVAL, "scan: staging does not fit in shared memory");
    uint64_t avail = (uint64_t)limit - staging - 64;
    if (a->smem_cap_bytes && a->smem_cap_bytes < avail) avail = a->smem_cap_bytes;
    uint32_t rows_fit = (uint32_t)(avail / (4ull * a->sigma));
    if (a->placement == AC_PLACE_GLOBAL) rows_fit = 0;
    uint32_t max_states = 0;
    for (auto &d : a->h_desc) max_states = std::max(max_states, d.states);
    const bool hybrid = max_states > rows_fit;
    if (a->placement == AC_PLACE_SMEM && hybrid)
        return set_error(AC_ERANGE, "scan: table of %u states does not fit in shared memory (%u rows)", max_states,
                         rows_fit);
    const uint32_t rows_used = std::min(max_states, rows_fit);
    p.smem_rows = rows_used;
    p.table_words = (rows_used * a->sigma + 3) & ~3u;
    const size_t smem = (size_t)p.table_words * 4 + staging;

    const bool acgt = t.fmt == AC_U8 && a->dna_acgt;
    KernelFn fn = pick_kernel(t.fmt, acgt, hybrid, cfg.chains);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(AC_ECUDA, "scan: %s", cudaGetErrorString(e));
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, a->device);
    uint64_t grid = cfg.ctas ? cfg.ctas : (uint64_t)sms;
    if (grid > p.num_tiles) grid = p.num_tiles;
    fn<<<(unsigned)grid, cfg.threads, smem, stream>>>(p);
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
