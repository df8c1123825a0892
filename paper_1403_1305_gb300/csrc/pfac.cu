// Scan with the failure-less machine (Section II.B, Figs. 2-4; the method
// of the paper's Section IV): a walk starts at every text position from the
// root and follows goto transitions until one is missing, producing the own
// patterns of every final state it passes. No failure function is built or
// used; the cost is one lookup per (start position, depth reached) instead of
// one per symbol, but every walk is short and independent of the others.
//
// GB300 mapping: persistent CTAs over tiles of start positions; a tile's text
// (its starts plus the longest pattern - 1 bytes after them) is copied into
// shared memory with 16-byte loads, the breadth-first prefix of the goto
// table (where every walk begins) sits in shared memory and deeper rows are
// read through L2; a warp's 32 walks advance together (the loop runs while
// any lane's walk is alive) so matches go through the same warp-aggregated
// emit as the folded-table scan.
#include "scan_kernel.cuh"

namespace acgb {
namespace kern {
namespace {

template <int MODE>
__device__ __forceinline__ uint32_t goto_lookup(const uint32_t *__restrict__ stab, const uint32_t *__restrict__ gtab,
                                                uint32_t hot, uint32_t sigma, uint32_t s, uint32_t c,
                                                uint64_t pol) {
    if (MODE == MODE_SMEM || s < hot) return stab[s * sigma + c];
    return ld_table(gtab + (uint64_t)s * sigma + c, pol);
}

template <int MODE>
__global__ void __launch_bounds__(512, 1) pfac_kernel(const __grid_constant__ ScanParams p, uint32_t tile_starts,
                                                      uint32_t span) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t lane = threadIdx.x & 31;
    uint32_t *stab = reinterpret_cast<uint32_t *>(smem);
    uint8_t *smap = smem + (((size_t)p.table_words * 4 + 127) & ~(size_t)127);
    uint8_t *stext = smap + 256;
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) smap[i] = p.sym_of_byte[i];
    const uint32_t sigma = p.sigma;
    const uint64_t n = p.nsym;
    const uint64_t pol = l2_evict_last();
    int cur_k = -1;
    for (uint64_t tile = blockIdx.x; tile < p.num_tiles; tile += gridDim.x) {
        const uint32_t k = (uint32_t)(tile % p.K);
        const uint64_t t0 = (tile / p.K) * tile_starts;
        const SubsetDev sd = p.subs[k];
        const uint32_t hot = min(sd.states, p.smem_rows);
        __syncthreads();  // every warp is done with the previous tile's text (and table)
        if ((int)k != cur_k) {
            const uint32_t words = hot * sigma;
            const uint4 *src4 = reinterpret_cast<const uint4 *>(sd.table);
            uint4 *dst4 = reinterpret_cast<uint4 *>(stab);
            for (uint32_t i = threadIdx.x; i < words / 4; i += blockDim.x) dst4[i] = __ldg(src4 + i);
            for (uint32_t i = (words & ~3u) + threadIdx.x; i < words; i += blockDim.x) stab[i] = __ldg(sd.table + i);
            cur_k = (int)k;
        }
        // the tile's text: bytes [t0, t0 + span), zero beyond the end of the text
        for (uint32_t i = threadIdx.x * 16; i < span; i += blockDim.x * 16) {
            if (t0 + i + 16 <= n) {
                *reinterpret_cast<uint4 *>(stext + i) = __ldg(reinterpret_cast<const uint4 *>(p.text + t0 + i));
            } else {
                for (uint32_t b = 0; b < 16; ++b) stext[i + b] = (t0 + i + b < n) ? p.text[t0 + i + b] : 0;
            }
        }
        __syncthreads();
        for (uint32_t r = 0; r < tile_starts; r += blockDim.x) {
            const uint64_t start = t0 + r + threadIdx.x;
            bool alive = start < n;
            uint32_t s = 0;
            uint64_t pos = start;
            while (__any_sync(kFull, alive)) {
                bool has = false;
                if (alive) {
                    if (pos >= n) {
                        alive = false;
                    } else {
                        const uint32_t c = smap[stext[pos - t0]];
                        const uint32_t e = c < sigma ? goto_lookup<MODE>(stab, sd.table, hot, sigma, s, c, pol) : kMissing;
                        if (e == kMissing) {
                            alive = false;
                        } else {
                            s = e & kStateMask;
                            has = (e & kFlag) != 0;
                        }
                    }
                }
                emit_warp(has, s, pos, 0, sd, p, lane);
                ++pos;
            }
        }
    }
}

}  // namespace
}  // namespace kern

int launch_pfac(const ac_automaton *a, const ScanText &t, const ScanOut &o, const ac_scan_config &cfg_in,
                cudaStream_t stream) {
    using namespace kern;
    if (t.fmt != AC_U8) return set_error(AC_EINVAL, "scan: the failure-less machine scans uint8 text only");
    if (t.n == 0) return AC_OK;
    const uint32_t threads = cfg_in.threads ? cfg_in.threads : 512;
    if (threads < 32 || threads > 512 || threads % 32)
        return set_error(AC_EINVAL, "scan: threads per CTA must be a multiple of 32 in [32, 512]");
    const uint32_t tile_starts = threads * 8;
    const uint32_t span = (tile_starts + a->max_len + 15) & ~15u;
    ScanParams p{};
    p.text = t.d_text;
    p.nbytes = t.n;
    p.nsym = t.n;
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
    p.num_tiles = ((t.n + tile_starts - 1) / tile_starts) * a->K;
    // shared memory: table prefix + map + the tile's text
    const int limit = scan_smem_limit(a->device);
    const uint64_t fixed = 256 + span + 256;
    if (fixed + 1152 > (uint64_t)limit) return set_error(AC_ERANGE, "scan: patterns too long for the failure-less scan");
    uint64_t avail = (uint64_t)limit - fixed - 128;  // the table is rounded up to 128 bytes
    if (a->smem_cap_bytes && a->smem_cap_bytes < avail) avail = a->smem_cap_bytes;
    uint32_t rows_fit = a->placement == AC_PLACE_GLOBAL ? 0u : (uint32_t)(avail / (4ull * a->sigma));
    uint32_t max_states = 0;
    for (auto &d : a->h_desc) max_states = std::max(max_states, d.states);
    const bool hybrid = max_states > rows_fit;
    if (a->placement == AC_PLACE_SMEM && hybrid)
        return set_error(AC_ERANGE, "scan: table of %u states does not fit in shared memory", max_states);
    p.smem_rows = std::min(max_states, rows_fit);
    p.table_words = (p.smem_rows * a->sigma + 3) & ~3u;
    const size_t smem = (((size_t)p.table_words * 4 + 127) & ~(size_t)127) + fixed;
    auto fn = hybrid ? pfac_kernel<MODE_HYBRID> : pfac_kernel<MODE_SMEM>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return set_error(AC_ECUDA, "scan: %s", cudaGetErrorString(e));
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, a->device);
    uint64_t grid = cfg_in.ctas ? cfg_in.ctas : (uint64_t)sms;
    if (grid > p.num_tiles) grid = p.num_tiles;
    fn<<<(unsigned)grid, threads, smem, stream>>>(p, tile_starts, span);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(AC_ECUDA, "scan launch: %s", cudaGetErrorString(e));
    return AC_OK;
}

}  // namespace acgb
