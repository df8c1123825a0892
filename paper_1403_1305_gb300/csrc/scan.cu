// Host side of the scan: launch planning (row geometry, tensor maps, shared
// memory), the small helper kernels (key padding, record conversion, error
// mark), and the radix sort of the match keys. The scan kernel itself is in
// scan_kernel.cuh (instantiated by the scan_k_*.cu translation units).
#include <cub/device/device_radix_sort.cuh>

#include "scan_kernel.cuh"
#include "scan_lean.cuh"
#include "scan_short.cuh"

namespace acgb {
using namespace kern;

namespace {

// A launch that, with `overlap`, may start before the launch ahead of it in
// the stream has finished (programmatic stream serialization; in a captured
// graph, a programmatic edge): the kernel calls pdl_wait() before it touches
// that launch's results. Without `overlap`, an ordinary launch.
template <typename... KArgs, typename... Args>
cudaError_t launch_overlapped(void (*fn)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              bool overlap, Args... args) {
    if (!overlap) {
        fn<<<grid, block, smem, s>>>(args...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, fn, args...);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// ------------------------------------------------------------------ small kernels
__global__ void fill_u64_kernel(unsigned long long *p, uint64_t count, unsigned long long value) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = value;
}

__global__ void zero3_kernel(unsigned long long *p0, uint64_t n0, unsigned long long *p1, uint64_t n1,
                             unsigned long long *p2, uint64_t n2) {
    kern::pdl_release();  // a scan or sort behind it may start; it waits for these writes
    kern::pdl_wait();     // launched overlapped: the launch before it (which may read these words) is done
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n0 + n1 + n2; i += stride) {
        if (i < n0) p0[i] = 0;
        else if (i < n0 + n1) p1[i - n0] = 0;
        else p2[i - n0 - n1] = 0;
    }
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
KernelFn pick_kernel(int fmt, bool acgt, int mode, uint32_t bx, uint32_t C, bool batch, bool track,
                     uint32_t stride = 1) {
    if (stride == 2) {  // single-text launches over ACGT bytes or packed text
        if (fmt == AC_PACKED2)
            return track ? kernels_packed_single_track_r2(mode, bx, C) : kernels_packed_single_plain_r2(mode, bx, C);
        return track ? kernels_u8_acgt_single_track_r2(mode, bx, C) : kernels_u8_acgt_single_plain_r2(mode, bx, C);
    }
    if (fmt == AC_PACKED2) return kernels_packed(batch, track, mode, bx, C);
    if (acgt) return kernels_u8_acgt(batch, track, mode, bx, C);
    return kernels_u8_map(batch, track, mode, bx, C);
}

// Estimated share of lookups at states beyond a shared-memory prefix of
// `rows` rows (the worst subset; tail masses are kept at powers of two, so
// the prefix is rounded down to one).
static double tail_beyond(const ac_automaton *a, uint32_t rows) {
    if (rows == 0) return 1.0;
    int k = 0;
    while (k < 31 && (1u << (k + 1)) <= rows) ++k;
    double worst = 0;
    for (auto &S : a->subs) worst = std::max(worst, S.tail_mass[k]);
    return worst;
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

// rows x row_bytes bytes at base, boxes of bx bytes x 32 rows. promote64:
// L2 fills of 64 bytes instead of 256 (many rows in flight at once: the
// promoted lines of every row must stay in L2 until their row reads them)
int encode_rows_map(CUtensorMap *m, const uint8_t *base, uint64_t row_bytes, uint64_t rows, uint32_t bx,
                    bool promote64 = false) {
    EncodeTiled enc = encoder();
    if (!enc) return set_error(AC_ECUDA, "scan: cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[2] = {row_bytes, rows};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {bx, 32};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     promote64 ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B : CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? AC_OK : set_error(AC_ECUDA, "scan: encoding the row tensor map failed (%d)", (int)r);
}

// bytes bytes at base, boxes of bx bytes
int encode_tail_map(CUtensorMap *m, const uint8_t *base, uint64_t bytes, uint32_t bx) {
    EncodeTiled enc = encoder();
    if (!enc) return set_error(AC_ECUDA, "scan: cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[1] = {bytes};
    cuuint64_t strides[1] = {0};
    cuuint32_t box[1] = {bx};
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
    const uint32_t bx = cfg.stage_bytes ? cfg.stage_bytes : kStageBytes;
    return 256 + 128 + 128 + warps * kNS * slot_bytes_for(cfg.chains, bx) + warps * kNS * 8;
}

// Bytes per chain row of a scan under cfg (a multiple of kStageBytes, at
// most the readable bytes rounded down to it; the text's row geometry).
uint64_t scan_row_bytes(const ac_scan_config &cfg, int fmt, uint64_t readable) {
    const uint32_t sym_per_byte = (fmt == AC_U8) ? 1 : 4;
    if (cfg.kernel == AC_KERNEL_SHORT) return short_row_bytes(cfg, fmt);
    uint64_t rb = ((uint64_t)cfg.row_len + sym_per_byte - 1) / sym_per_byte;
    rb = (rb + kStageBytes - 1) / kStageBytes * kStageBytes;
    if (rb > (1u << 24)) rb = 1u << 24;
    const uint64_t rmax = readable / kStageBytes * kStageBytes;
    if (rb > rmax) rb = rmax;
    if (rb == 0) rb = kStageBytes;
    return rb;
}

// ------------------------------------------------------------------ lean kernel
bool lean_shape_ok(uint32_t threads, uint32_t chains) {
    return (threads == 1024 && (chains == 4 || chains == 3 || chains == 2)) || (threads == 768 && chains == 4) ||
           (threads == 512 && chains == 4);
}

// Why the lean kernel cannot scan format fmt of `a` under configuration c
// (threads/chains 0 = its defaults), or nullptr when it can.
const char *lean_unfit(const ac_automaton *a, const ac_scan_config &c, int fmt) {
    if (a->machine != AC_MACHINE_DFA) return "it walks the folded machine only";
    if (a->sigma != 4 || !(fmt == AC_PACKED2 || (fmt == AC_U8 && a->dna_acgt)))
        return "it needs a 4-letter machine and ACGT bytes or packed text";
    if (c.stride == 2) return "it uses the one-symbol table (stride 1)";
    if (a->placement != AC_PLACE_AUTO && a->placement != AC_PLACE_SMEM && a->placement != AC_PLACE_HYBRID16)
        return "it supports placements AUTO, SMEM and HYBRID16";
    if (c.stage_bytes && c.stage_bytes != kern::kLeanBX) return "it uses 16-byte stages";
    const uint32_t t = c.threads ? c.threads : 1024;
    const uint32_t ch = c.chains ? c.chains : (fmt == AC_U8 ? 2u : 3u);
    if (!lean_shape_ok(t, ch))
        return "(threads, chains) must be (1024, 4), (1024, 3), (1024, 2), (768, 4) or (512, 4)";
    uint32_t max_states = 0;
    for (auto &d : a->h_desc) {
        if (d.states >= (1u << 28)) return "it needs fewer than 2^28 states per subset";
        if (!d.table_e16) return "the escape-coded 16-bit prefix is missing";
        max_states = std::max(max_states, d.states);
    }
    if (a->placement == AC_PLACE_SMEM) {
        const int limit = scan_smem_limit(a->device);
        uint64_t room = (uint64_t)std::max(0, limit - (int)kern::lean_stage_bytes(t, ch) - 128);
        if (a->smem_cap_bytes && a->smem_cap_bytes < room) room = a->smem_cap_bytes;
        if (c.smem_table_bytes && c.smem_table_bytes < room) room = c.smem_table_bytes;
        if ((uint64_t)max_states * 16 > room) return "the whole table does not fit its shared memory";
    }
    return nullptr;
}

// Row bytes of a short-text scan: row_len symbols rounded up to 16-byte
// words, one to four words (default one).
uint32_t short_row_bytes(const ac_scan_config &cfg, int fmt) {
    const uint64_t spb = (fmt == AC_U8) ? 1 : 4;
    uint64_t rb = cfg.row_len ? ((uint64_t)cfg.row_len + spb - 1) / spb : 16;
    rb = (rb + 15) / 16 * 16;
    return (uint32_t)std::min<uint64_t>(rb, kShortMaxRowBytes);
}

// Why the short-text kernel cannot scan format fmt of `a` under
// configuration c, or nullptr when it can.
const char *short_unfit(const ac_automaton *a, const ac_scan_config &c, int fmt) {
    if (a->machine != AC_MACHINE_DFA) return "it walks the folded machine only";
    if (a->K != 1) return "it scans one machine (no pattern subsets)";
    if (a->sigma != 4) return "it needs a 4-letter machine";
    if (c.stride == 2) return "it uses the one-symbol table (stride 1)";
    if (a->placement != AC_PLACE_AUTO && a->placement != AC_PLACE_SMEM && a->placement != AC_PLACE_HYBRID16)
        return "it supports placements AUTO, SMEM and HYBRID16";
    if (c.chains > 1) return "it runs one chain per thread";
    if (c.threads && (c.threads < 64 || c.threads > 1024 || c.threads % 32))
        return "threads per CTA must be a multiple of 32 in [64, 1024]";
    const uint64_t spb = (fmt == AC_U8) ? 1 : 4;
    if (c.row_len && (c.row_len + spb - 1) / spb > kShortMaxRowBytes) return "rows are at most 64 bytes of text";
    if (a->h_desc.empty() || a->h_desc[0].states >= (1u << 28)) return "it needs fewer than 2^28 states";
    const uint64_t warm_bytes = (fmt == AC_U8) ? a->h_desc[0].warm : (a->h_desc[0].warm + 3ull) / 4;
    if ((warm_bytes + 15) / 16 + short_row_bytes(c, fmt) / 16 > kern::kShortMaxWords)
        return "the warm-up (longest pattern - 1 symbols) and the row exceed nine 16-byte words";
    return nullptr;
}

static void fill_config(const ac_automaton *a, ac_scan_config c, uint64_t n, int fmt, ac_scan_config *cfg);

// Would the general kernel's automatic plan use two symbols per lookup for
// format fmt (the two-symbol table beats the lean one-symbol scan there)?
static bool general_picks_stride2(const ac_automaton *a, int fmt) {
    if (!a->has_table2 || scan_stride(a, fmt, 0) != 2) return false;
    ac_scan_config base{}, g{};
    base.kernel = AC_KERNEL_GENERAL;
    fill_config(a, base, 1, fmt, &g);
    ScanPlan plan{};
    return plan_scan(a, g, fmt, &plan) == AC_OK && plan.stride == 2;
}

void default_config(const ac_automaton *a, uint64_t n, int fmt, ac_scan_config *cfg) {
    fill_config(a, a->cfg, n, fmt, cfg);
}

// The configuration a scan of n symbols (format fmt) runs with, from the
// configuration c whose zero fields take their defaults.
static void fill_config(const ac_automaton *a, ac_scan_config c, uint64_t n, int fmt, ac_scan_config *cfg) {
    const ac_scan_config given = c;
    // a short text on one 4-letter machine: one thread per 16-byte row, each
    // thread's window loaded in one round trip (the pipelined kernels pay a
    // copy round trip per 16-byte stage and leave most of the GPU idle)
    const uint64_t nbytes = (fmt == AC_U8) ? n : (n + 3) / 4;
    const bool untouched = !c.row_len && !c.threads && !c.chains && !c.ctas && !c.stage_bytes;
    if (a->device >= 0 &&
        (c.kernel == AC_KERNEL_SHORT ||
         (c.kernel == AC_KERNEL_AUTO && untouched && n <= kShortAutoSymbols && !short_unfit(a, c, fmt)))) {
        // (values given for the short kernel stay as they are: the launch refuses those it cannot run)
        c.kernel = AC_KERNEL_SHORT;
        if (!c.threads) c.threads = 512;
        if (!c.chains) c.chains = 1;
        if (!c.stride) c.stride = 1;
        if (!c.row_len) {
            // about kShortRows rows (the GPU holds ~300k threads): rows of 16
            // bytes while the text is short (each thread's walk, mostly
            // warm-up, is the latency), longer ones as it grows (fewer warm-up
            // lookups in all); warm-up and row within the window
            const uint64_t warm_bytes =
                a->h_desc.empty() ? 0 : (fmt == AC_U8 ? a->h_desc[0].warm : (a->h_desc[0].warm + 3ull) / 4);
            const uint64_t words_left = kern::kShortMaxWords - std::min<uint64_t>(kern::kShortMaxWords - 1,
                                                                                  (warm_bytes + 15) / 16);
            uint64_t rb = (nbytes / kShortRows + 15) / 16 * 16;
            rb = std::min<uint64_t>(std::max<uint64_t>(rb, 16), std::min<uint64_t>(kShortMaxRowBytes, 16 * words_left));
            c.row_len = (uint32_t)rb * (fmt == AC_U8 ? 1 : 4);
        }
        *cfg = c;
        return;
    }
    const bool lean_ok = c.kernel != AC_KERNEL_GENERAL && a->device >= 0 && !lean_unfit(a, c, fmt) &&
                         !(c.kernel == AC_KERNEL_AUTO && c.stride == 0 && general_picks_stride2(a, fmt));
    if (lean_ok) {
        c.kernel = AC_KERNEL_LEAN;
        if (!c.threads) c.threads = 1024;
        // byte text: 2 chains per thread (less staging, so a larger shared-
        // memory prefix, and the row block ends sooner); packed text: 3 (a
        // 16-byte stage is 64 symbols)
        if (!c.chains) c.chains = fmt == AC_U8 ? 2 : 3;
        c.stage_bytes = kern::kLeanBX;
        if (!c.row_len) {
            int sms = 148;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, a->device);
            const uint64_t chains = (uint64_t)sms * c.threads * c.chains;
            uint64_t want = (n + chains - 1) / chains;
            // one machine: all chains busy, rows down to one 32-byte block (a
            // short text spreads over the SMs and each warp's walk is short);
            // subset machines: the general kernel's rule
            const uint64_t block = fmt == AC_U8 ? 32 : 128;
            const uint64_t lo = a->K == 1 ? block : std::max<uint64_t>(256, 8ull * a->max_len);
            uint64_t L = std::max<uint64_t>(want, lo);
            if (L > (1u << 20)) L = 1u << 20;
            c.row_len = (uint32_t)L;
        }
        *cfg = c;
        return;
    }
    if (c.kernel == AC_KERNEL_AUTO) c.kernel = AC_KERNEL_GENERAL;
    if (!c.threads) c.threads = 512;
    if (!c.chains) c.chains = 2;
    // 16-byte stages leave more shared memory to the table and double the
    // stages in flight; with many small subset tables (which fit in shared
    // memory anyway) 32-byte stages do fewer pipeline round trips
    if (!c.stage_bytes) c.stage_bytes = (a->K >= 4 || c.chains == 1) ? 32 : 16;
    if (!c.smem_table_bytes && a->sigma >= 16) {
        // a large-alphabet table that does not fit: keep a small prefix in shared
        // memory and leave the rest of the SRAM to L1, which follows the text's
        // letter skew better than a fixed breadth-first prefix
        uint64_t biggest = 0;
        for (auto &d : a->h_desc) biggest = std::max<uint64_t>(biggest, (uint64_t)d.states * a->sigma * 4);
        if (biggest > (160u << 10)) c.smem_table_bytes = 16u << 10;
    }
    if (!given.chains && a->device >= 0 && a->machine == AC_MACHINE_DFA) {
        // with the 16-bit prefix (a large 4-letter machine) most steps still
        // wait on L2 for some lane: 4 chains per thread keep more in flight
        ScanPlan plan{};
        if (plan_scan(a, c, fmt, &plan) == AC_OK && plan.mode == kern::MODE_H16) {
            c.chains = 4;
            if (!given.stage_bytes) c.stage_bytes = 16;
        }
    }
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

uint32_t scan_stride(const ac_automaton *a, int fmt, uint32_t want) {
    if (want == 1 || !a->has_table2) return 1;
    const bool format_ok = fmt == AC_PACKED2 || (fmt == AC_U8 && a->dna_acgt);
    if (want == 2) return format_ok ? 2 : 0;  // 0: asked for but not possible
    return format_ok ? 2 : 1;
}

// Lean plan: every row in shared memory (32-bit row offsets) when the
// largest subset fits, else the longest escape-coded 16-bit prefix that fits.
static int plan_lean(const ac_automaton *a, const ac_scan_config &cfg, int fmt, ScanPlan *out) {
    if (const char *why = lean_unfit(a, cfg, fmt)) return set_error(AC_EINVAL, "scan: lean kernel: %s", why);
    const int limit = scan_smem_limit(a->device);
    const uint32_t staging = kern::lean_stage_bytes(cfg.threads, cfg.chains);
    if ((int)staging + 1024 > limit) return set_error(AC_EINVAL, "scan: lean staging does not fit in shared memory");
    uint64_t avail = (uint64_t)limit - staging - 128;
    if (a->smem_cap_bytes && a->smem_cap_bytes < avail) avail = a->smem_cap_bytes;
    if (cfg.smem_table_bytes && cfg.smem_table_bytes < avail) avail = cfg.smem_table_bytes;
    uint32_t max_states = 0, max_rows_e16 = 0;
    for (auto &d : a->h_desc) {
        max_states = std::max(max_states, d.states);
        max_rows_e16 = std::max(max_rows_e16, d.rows_e16);
    }
    ScanPlan pl{};
    pl.lean = true;
    pl.stride = 1;
    if ((uint64_t)max_states * 16 <= avail && a->placement != AC_PLACE_HYBRID16) {
        pl.mode = kern::LEAN_SMEM32;
        pl.smem_rows = max_states;
        pl.table_words = max_states * 4;
    } else {
        if (a->placement == AC_PLACE_SMEM)
            return set_error(AC_ERANGE, "scan: table of %u states does not fit in shared memory", max_states);
        pl.mode = kern::LEAN_E16;
        pl.smem_rows = (uint32_t)std::min<uint64_t>(max_rows_e16, avail / 8);
        pl.table_words = (pl.smem_rows * 2 + 3) & ~3u;
    }
    pl.smem = (((size_t)pl.table_words * 4 + 127) & ~(size_t)127) + staging;
    if (pl.smem > (size_t)limit) return set_error(AC_EINVAL, "scan: lean shared memory plan exceeds the limit");
    *out = pl;
    return AC_OK;
}

// Short-text plan: the whole table in shared memory when it fits in the
// room that leaves two CTAs per SM (all of the SM's room with placement
// SMEM), else the longest escape-coded 16-bit prefix that fits there.
static int plan_short(const ac_automaton *a, const ac_scan_config &cfg, int fmt, ScanPlan *out) {
    if (const char *why = short_unfit(a, cfg, fmt)) return set_error(AC_EINVAL, "scan: short-text kernel: %s", why);
    const int limit = scan_smem_limit(a->device);
    uint64_t room = (uint64_t)std::max(0, limit - 512);
    if (a->placement != AC_PLACE_SMEM) room = std::min<uint64_t>(room, kShortSmemBytes);
    if (a->smem_cap_bytes && a->smem_cap_bytes < room) room = a->smem_cap_bytes;
    if (cfg.smem_table_bytes && cfg.smem_table_bytes < room) room = cfg.smem_table_bytes;
    const SubsetDev &d = a->h_desc[0];
    ScanPlan pl{};
    pl.short_text = true;
    pl.stride = 1;
    if ((uint64_t)d.states * 16 <= room && a->placement != AC_PLACE_HYBRID16) {
        pl.mode = kern::SHORT_FULL;
        pl.smem_rows = d.states;
        pl.table_words = d.states * 4;
    } else {
        if (a->placement == AC_PLACE_SMEM)
            return set_error(AC_ERANGE, "scan: table of %u states does not fit in shared memory", d.states);
        if (!d.table_e16) return set_error(AC_EINVAL, "scan: short-text kernel: the 16-bit prefix is missing");
        pl.mode = kern::SHORT_E16;
        pl.smem_rows = (uint32_t)std::min<uint64_t>(d.rows_e16, room / 8);
        pl.table_words = (pl.smem_rows * 2 + 3) & ~3u;
    }
    pl.smem = (size_t)pl.table_words * 4 + 256;
    *out = pl;
    return AC_OK;
}

int plan_scan(const ac_automaton *a, const ac_scan_config &cfg, int fmt, ScanPlan *out) {
    if (cfg.kernel == AC_KERNEL_SHORT) return plan_short(a, cfg, fmt, out);
    if (cfg.kernel == AC_KERNEL_LEAN) return plan_lean(a, cfg, fmt, out);
    uint32_t max_states = 0, max_rows16 = 0;
    bool has16 = a->sigma == 4 && !a->h_desc.empty();
    for (auto &d : a->h_desc) {
        max_states = std::max(max_states, d.states);
        max_rows16 = std::max(max_rows16, d.rows16);
        has16 = has16 && d.table16 && d.rows16 > 0;
    }
    uint32_t stride = scan_stride(a, fmt, cfg.stride);
    if (stride == 0)
        return set_error(AC_EINVAL, "scan: stride 2 needs the two-symbol table and ACGT bytes or packed text");
    const uint32_t bx = cfg.stage_bytes ? cfg.stage_bytes : kStageBytes;
    const uint32_t sym_per_stage = fmt == AC_U8 ? bx : 4 * bx;
    ScanPlan one{}, two{};
    bool hyb = false;
    const int rc1 = plan_smem(a->device, cfg, a->sigma, a->placement, a->smem_cap_bytes, max_states, &one.smem_rows,
                              &hyb, &one.smem, &one.table_words);
    one.mode = hyb ? MODE_HYBRID : MODE_SMEM;
    one.stride = 1;
    if (stride == 2) {
        bool hyb2 = false;
        const int rc2 = plan_smem(a->device, cfg, 16, a->placement, a->smem_cap_bytes, max_states, &two.smem_rows,
                                  &hyb2, &two.smem, &two.table_words);
        two.mode = hyb2 ? MODE_HYBRID : MODE_SMEM;
        two.stride = 2;
        if (cfg.stride == 2) {
            if (rc2) return rc2;
            *out = two;
            return AC_OK;
        }
        // automatic: two symbols per lookup pay when the one-symbol table
        // overflows shared memory and the two-symbol prefix still holds
        // nearly every state a walk visits
        if (rc2 == AC_OK && rc1 == AC_OK && hyb && tail_beyond(a, two.smem_rows) <= 0.02) {
            *out = two;
            return AC_OK;
        }
    }
    if (rc1) return rc1;
    *out = one;
    if (!hyb || one.smem_rows == 0 || (cfg.chains != 2 && cfg.chains != 4)) return AC_OK;
    const int place = a->placement;
    uint32_t rows_pow2 = 1;
    while (rows_pow2 * 2 <= one.smem_rows) rows_pow2 *= 2;
    if (place == AC_PLACE_OPT ||
        (place == AC_PLACE_AUTO && tail_beyond(a, rows_pow2) * (32.0 * cfg.chains * sym_per_stage) < 0.01)) {
        // MODE_OPT pays when a warp's stage rarely reaches a state beyond the
        // power-of-two prefix (expected stages walked again below 1%)
        out->mode = MODE_OPT;
        out->smem_rows = rows_pow2;
        out->table_words = (rows_pow2 * a->sigma + 3) & ~3u;
        out->smem = (((size_t)out->table_words * 4 + 127) & ~(size_t)127) + scan_stage_bytes_per_cta(cfg);
        return AC_OK;
    }
    if (has16 && (place == AC_PLACE_HYBRID16 || place == AC_PLACE_AUTO)) {
        ScanPlan h{};
        bool unused = false;
        if (plan_smem(a->device, cfg, 2, AC_PLACE_AUTO, a->smem_cap_bytes, max_rows16, &h.smem_rows, &unused,
                      &h.smem, &h.table_words) == AC_OK &&
            h.smem_rows > 0) {
            double m16 = 0;
            for (auto &d : a->h_desc) {
                const uint32_t staged = std::min(d.rows16, h.smem_rows);
                int k = 0;
                while (k < 31 && (1u << (k + 1)) <= staged) ++k;
                const auto &S = a->subs[&d - a->h_desc.data()];
                m16 = std::max(m16, staged ? S.tail_mass[k] : 1.0);
            }
            // the 16-bit lookup costs a little more per step: worth it when the
            // 32-bit prefix leaves many lookups to L2 and the 16-bit one far fewer
            const double m32 = tail_beyond(a, one.smem_rows);
            if (place == AC_PLACE_HYBRID16 || (m32 >= 0.05 && m16 < 0.5 * m32)) {
                h.mode = MODE_H16;
                h.stride = 1;
                *out = h;
            }
        }
    }
    return AC_OK;
}

int key_shift_for(const ac_automaton *a) { return (int)bits_for(a->P ? a->P - 1 : 0); }

// One folded machine: every match at a position is emitted by the one chain
// that owns the position, as its state's output (ids ascending) into
// consecutive slots, so a stable sort by the position bits alone orders the
// keys. Subsets and the failure-less machine emit a position's matches from
// several chains: the whole key is sorted.
int sort_begin_bit(const ac_automaton *a) {
    return (a->machine == AC_MACHINE_DFA && a->K == 1) ? key_shift_for(a) : 0;
}

int plan_smem(int device, const ac_scan_config &cfg, uint32_t sigma, int placement, uint32_t smem_cap,
              uint32_t max_states, uint32_t *rows_used, bool *hybrid, size_t *smem_bytes, uint32_t *table_words) {
    // shared memory: table prefix (rounded to 128 bytes) + map + staging + barriers
    const int limit = scan_smem_limit(device);
    const uint32_t staging = scan_stage_bytes_per_cta(cfg);
    if ((int)staging + 1024 > limit) return set_error(AC_EINVAL, "scan: staging does not fit in shared memory");
    uint64_t avail = (uint64_t)limit - staging - 128;
    if (smem_cap && smem_cap < avail) avail = smem_cap;
    if (cfg.smem_table_bytes && cfg.smem_table_bytes < avail) avail = cfg.smem_table_bytes;
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
    if ((cfg.stage_bytes && cfg.stage_bytes != 16 && cfg.stage_bytes != 32) || (cfg.stage_bytes == 16 && cfg.chains == 1))
        return set_error(AC_EINVAL, "batch: bad stage bytes");
    if (b.num_tiles == 0) return AC_OK;
    if (b.row_bytes % kStageBytes || ((uintptr_t)b.arena & 15))
        return set_error(AC_EINVAL, "batch: arena rows must be 32-byte multiples at a 16-byte aligned address");
    ScanParams p{};
    p.text = b.arena;
    p.nbytes = b.rows * b.row_bytes;
    p.nsym = 0;
    p.full_rows = b.rows;
    p.num_rows = b.rows;
    p.row_begin = 0;
    p.row_end = b.rows;
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
    p.wait_ns = wait_limit_ns();
    p.key_shift = b.key_shift;
    p.tail_bytes = 0;
    p.items = b.items;
    p.tiles = b.tiles;
    p.num_items = b.num_items;
    memcpy(p.sym_of_byte, b.sym_of_byte, 256);
    if (b.rows >= (1ull << 31)) return set_error(AC_ERANGE, "batch: arena too large for one launch");
    CUtensorMap rows_map, tail_map;
    memset(&tail_map, 0, sizeof(tail_map));
    const uint32_t bx = cfg.stage_bytes ? cfg.stage_bytes : kStageBytes;
    int rc = encode_rows_map(&rows_map, b.arena, b.row_bytes, b.rows, bx);
    if (rc) return rc;
    uint32_t rows_used = 0;
    bool hybrid = false;
    size_t smem = 0;
    rc = plan_smem(b.device, cfg, b.sigma, b.placement, b.smem_cap_bytes, b.max_states, &rows_used, &hybrid, &smem,
                   &p.table_words);
    if (rc) return rc;
    p.smem_rows = rows_used;
    KernelFn fn = pick_kernel(b.fmt, b.fmt == AC_U8 && b.acgt, hybrid ? MODE_HYBRID : MODE_SMEM, bx, cfg.chains, true,
                              b.track_flags != 0);
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

// The lean kernel (scan_lean.cuh): one-symbol scan of ACGT bytes or packed text.
static int launch_lean(const ac_automaton *a, const ScanText &t, const ScanOut &o, const ac_scan_config &cfg,
                       cudaStream_t stream) {
    const uint64_t nbytes = (t.fmt == AC_U8) ? t.n : (t.n + 3) / 4;
    if (nbytes == 0) return AC_OK;
    const uint64_t readable = std::max(nbytes, t.readable);
    if (readable < kStageBytes) return set_error(AC_EINVAL, "scan: text buffer shorter than one stage");
    if ((uintptr_t)t.d_text & 15) return set_error(AC_EINVAL, "scan: text must be 16-byte aligned");
    ScanPlan plan{};
    int rc = plan_lean(a, cfg, t.fmt, &plan);
    if (rc) return rc;
    const uint64_t rb = scan_row_bytes(cfg, t.fmt, readable);

    ScanParams p{};
    p.text = t.d_text;
    p.nbytes = nbytes;
    p.nsym = t.n;
    p.row_bytes = (uint32_t)rb;
    p.full_rows = readable / rb;
    const uint64_t covered = p.full_rows * rb;
    p.tail_bytes = nbytes > covered ? (uint32_t)(nbytes - covered) : 0u;
    p.num_rows = p.full_rows + (p.tail_bytes ? 1 : 0);
    p.row_begin = std::min(t.row_begin, p.num_rows);
    p.row_end = t.row_end ? std::min(t.row_end, p.num_rows) : p.num_rows;
    if (p.row_end <= p.row_begin) return AC_OK;
    p.rows_per_tile = cfg.threads * cfg.chains;
    p.K = a->K;
    p.sigma = a->sigma;
    p.subs = a->d_desc;
    p.keys = o.keys;
    p.cap = o.cap;
    p.num = o.num;
    p.counts = o.counts;
    p.err = o.err;
    p.wait_ns = wait_limit_ns();
    p.key_shift = (uint32_t)key_shift_for(a);
    p.smem_rows = plan.smem_rows;
    p.table_words = plan.table_words;
    memcpy(p.sym_of_byte, a->sym_of_byte, 256);
    const uint64_t row_blocks = (p.row_end - p.row_begin + p.rows_per_tile - 1) / p.rows_per_tile;
    p.num_tiles = row_blocks * a->K;
    if (p.full_rows >= (1ull << 31) || p.num_rows * rb >= (1ull << 40))
        return set_error(AC_ERANGE, "scan: text too long for the row tensor map");

    CUtensorMap rows_map, tail_map;
    memset(&rows_map, 0, sizeof(rows_map));
    memset(&tail_map, 0, sizeof(tail_map));
    rc = encode_rows_map(&rows_map, t.d_text, rb, p.full_rows, kern::kLeanBX, true);
    if (rc) return rc;
    if (p.tail_bytes) {
        rc = encode_tail_map(&tail_map, t.d_text + covered, p.tail_bytes, kern::kLeanBX);
        if (rc) return rc;
    }
    kern::LeanFn fn = nullptr;
    if (t.fmt == AC_PACKED2)
        fn = plan.mode == kern::LEAN_SMEM32 ? kern::lean_packed_smem32(cfg.threads, cfg.chains)
                                            : kern::lean_packed_e16(cfg.threads, cfg.chains);
    else
        fn = plan.mode == kern::LEAN_SMEM32 ? kern::lean_u8_smem32(cfg.threads, cfg.chains)
                                            : kern::lean_u8_e16(cfg.threads, cfg.chains);
    if (!fn) return set_error(AC_EINVAL, "scan: no lean kernel for this configuration");
    if (o.q && o.q_cap) {
        p.q = o.q;
        p.q_cap = o.q_cap;
    }
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
    if (e != cudaSuccess) return set_error(AC_ECUDA, "scan: %s", cudaGetErrorString(e));
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, a->device);
    // one machine: warps take blocks of 32 * chains rows, so a CTA needs only
    // one block; subset machines: CTA tiles of threads * chains rows
    const uint64_t units =
        a->K == 1 ? (p.row_end - p.row_begin + 32ull * cfg.chains - 1) / (32ull * cfg.chains) : p.num_tiles;
    uint64_t grid = cfg.ctas ? cfg.ctas : (uint64_t)sms;
    if (grid > units) grid = units;
    fn<<<(unsigned)grid, cfg.threads, plan.smem, stream>>>(p, rows_map, tail_map);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(AC_ECUDA, "scan launch: %s", cudaGetErrorString(e));
    return AC_OK;
}

// One thread per row of rb bytes; rows [row_begin, row_end) of ceil(bytes / rb).
static int launch_short(const ac_automaton *a, const ScanText &t, const ScanOut &o, const ac_scan_config &cfg,
                        cudaStream_t stream) {
    const uint64_t nbytes = (t.fmt == AC_U8) ? t.n : (t.n + 3) / 4;
    if (nbytes == 0) return AC_OK;
    if ((uintptr_t)t.d_text & 15) return set_error(AC_EINVAL, "scan: text must be 16-byte aligned");
    ScanPlan plan{};
    int rc = plan_short(a, cfg, t.fmt, &plan);
    if (rc) return rc;
    const uint32_t rb = short_row_bytes(cfg, t.fmt);
    const uint32_t threads = cfg.threads ? cfg.threads : 512;

    ScanParams p{};
    p.text = t.d_text;
    p.nbytes = nbytes;
    p.nsym = t.n;
    p.row_bytes = rb;
    p.num_rows = (nbytes + rb - 1) / rb;
    p.full_rows = nbytes / rb;
    p.row_begin = std::min(t.row_begin, p.num_rows);
    p.row_end = t.row_end ? std::min(t.row_end, p.num_rows) : p.num_rows;
    if (p.row_end <= p.row_begin) return AC_OK;
    p.K = 1;
    p.sigma = a->sigma;
    p.subs = a->d_desc;
    p.sub0 = a->h_desc[0];
    p.keys = o.keys;
    p.cap = o.cap;
    p.num = o.num;
    p.counts = o.counts;
    p.err = o.err;
    p.key_shift = (uint32_t)key_shift_for(a);
    p.smem_rows = plan.smem_rows;
    p.table_words = plan.table_words;
    memcpy(p.sym_of_byte, a->sym_of_byte, 256);
    const uint64_t grid = (p.row_end - p.row_begin + threads - 1) / threads;
    if (grid >= (1ull << 31)) return set_error(AC_ERANGE, "scan: text too long for the short-text kernel");
    const uint64_t warm_bytes = (t.fmt == AC_U8) ? a->h_desc[0].warm : (a->h_desc[0].warm + 3ull) / 4;
    const uint32_t words = (uint32_t)((warm_bytes + 15) / 16 + rb / 16);
    kern::ShortFn fn = t.fmt == AC_PACKED2 ? (plan.mode == kern::SHORT_FULL ? kern::short_packed_full(words)
                                                                            : kern::short_packed_e16(words))
                                           : (plan.mode == kern::SHORT_FULL ? kern::short_u8_full(words, a->dna_acgt)
                                                                            : kern::short_u8_e16(words, a->dna_acgt));
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
    if (e != cudaSuccess) return set_error(AC_ECUDA, "scan: %s", cudaGetErrorString(e));
    e = launch_overlapped(fn, dim3((unsigned)grid), dim3(threads), plan.smem, stream, o.after_zero, p);
    if (e != cudaSuccess) return set_error(AC_ECUDA, "scan launch: %s", cudaGetErrorString(e));
    return AC_OK;
}

int launch_scan(const ac_automaton *a, const ScanText &t, const ScanOut &o, const ac_scan_config &cfg_in,
                cudaStream_t stream) {
    if (a->machine == AC_MACHINE_PFAC) return launch_pfac(a, t, o, cfg_in, stream);
    if (cfg_in.kernel == AC_KERNEL_SHORT) return launch_short(a, t, o, cfg_in, stream);
    if (cfg_in.kernel == AC_KERNEL_LEAN) return launch_lean(a, t, o, cfg_in, stream);
    ac_scan_config cfg = cfg_in;
    if (cfg.threads < 32 || cfg.threads > 512 || cfg.threads % 32)
        return set_error(AC_EINVAL, "scan: threads per CTA must be a multiple of 32 in [32, 512]");
    if (cfg.chains != 1 && cfg.chains != 2 && cfg.chains != 4)
        return set_error(AC_EINVAL, "scan: chains per thread must be 1, 2 or 4");
    if (cfg.stage_bytes && cfg.stage_bytes != 16 && cfg.stage_bytes != 32)
        return set_error(AC_EINVAL, "scan: stage bytes must be 16 or 32");
    if (cfg.stage_bytes == 16 && cfg.chains == 1)
        return set_error(AC_EINVAL, "scan: 16-byte stages need 2 or 4 chains per thread");
    const uint64_t nbytes = (t.fmt == AC_U8) ? t.n : (t.n + 3) / 4;
    if (nbytes == 0) return AC_OK;
    const uint64_t readable = std::max(nbytes, t.readable);
    if (readable < kStageBytes) return set_error(AC_EINVAL, "scan: text buffer shorter than one stage");
    if ((uintptr_t)t.d_text & 15) return set_error(AC_EINVAL, "scan: text must be 16-byte aligned");
    const uint64_t rb = scan_row_bytes(cfg, t.fmt, readable);

    ScanParams p{};
    p.text = t.d_text;
    p.nbytes = nbytes;
    p.nsym = t.n;
    p.row_bytes = (uint32_t)rb;
    p.full_rows = readable / rb;
    const uint64_t covered = p.full_rows * rb;
    p.tail_bytes = nbytes > covered ? (uint32_t)(nbytes - covered) : 0u;
    p.num_rows = p.full_rows + (p.tail_bytes ? 1 : 0);
    p.row_begin = std::min(t.row_begin, p.num_rows);
    p.row_end = t.row_end ? std::min(t.row_end, p.num_rows) : p.num_rows;
    if (p.row_end <= p.row_begin) return AC_OK;
    p.rows_per_tile = cfg.threads * cfg.chains;
    p.K = a->K;
    p.sigma = a->sigma;
    p.subs = a->d_desc;
    p.keys = o.keys;
    p.cap = o.cap;
    p.num = o.num;
    p.counts = o.counts;
    p.err = o.err;
    p.wait_ns = wait_limit_ns();
    p.key_shift = (uint32_t)key_shift_for(a);
    memcpy(p.sym_of_byte, a->sym_of_byte, 256);
    const uint64_t row_blocks = (p.row_end - p.row_begin + p.rows_per_tile - 1) / p.rows_per_tile;
    p.num_tiles = row_blocks * a->K;
    if (p.full_rows >= (1ull << 31) || p.num_rows * rb >= (1ull << 40))
        return set_error(AC_ERANGE, "scan: text too long for the row tensor map");

    CUtensorMap rows_map, tail_map;
    memset(&rows_map, 0, sizeof(rows_map));
    memset(&tail_map, 0, sizeof(tail_map));
    const uint32_t bx = cfg.stage_bytes ? cfg.stage_bytes : kStageBytes;
    int rc = encode_rows_map(&rows_map, t.d_text, rb, p.full_rows, bx);
    if (rc) return rc;
    if (p.tail_bytes) {
        rc = encode_tail_map(&tail_map, t.d_text + covered, p.tail_bytes, bx);
        if (rc) return rc;
    }

    ScanPlan plan{};
    rc = plan_scan(a, cfg, t.fmt, &plan);
    if (rc) return rc;
    p.smem_rows = plan.smem_rows;
    p.table_words = plan.table_words;
    const size_t smem = plan.smem;
    const int mode = plan.mode;
    const uint32_t stride = plan.stride;

    const bool acgt = t.fmt == AC_U8 && a->dna_acgt;
    // one machine holding the whole pattern set: matches are frequent enough
    // for flag tracking to pay; many subset machines: keep the loop lean
    KernelFn fn = pick_kernel(t.fmt, acgt, mode, bx, cfg.chains, false, a->K < 4, stride);
    if (!fn) return set_error(AC_EINVAL, "scan: no kernel for this configuration");
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

int launch_zero(unsigned long long *p0, uint64_t n0, unsigned long long *p1, uint64_t n1, unsigned long long *p2,
                uint64_t n2, cudaStream_t stream, bool overlap) {
    const uint64_t total = n0 + n1 + n2;
    if (!total) return AC_OK;
    const uint64_t blocks = std::min<uint64_t>((total + 255) / 256, 1024);
    cudaError_t e = launch_overlapped(zero3_kernel, dim3((unsigned)blocks), dim3(256), 0, stream, overlap, p0, n0, p1,
                                      n1, p2, n2);
    return e == cudaSuccess ? AC_OK : set_error(AC_ECUDA, "zero: %s", cudaGetErrorString(e));
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

// Up to kSmallSortMax keys, sorted by rank: keys are distinct (one
// (position, pattern) pair each), so a key's place in the sorted order is the
// number of keys below it and each key is written straight there -- one
// launch, no digit passes. A CTA copies all the keys into shared memory
// (asynchronous 16-byte copies; the first kRankEarly are requested before the
// key count has arrived, so a short list costs one round trip) and ranks 32 of them: a thread
// holds 4 keys and counts the keys below them in one of 64 interleaved slices
// of the key array (read 16 bytes at once, each read serving 8 comparisons);
// the slices' counts are summed with shuffles and then across the two warps
// of a slice group. The records are the (position, id) pairs of the keys.
namespace {
constexpr uint32_t kRankKeys = 32, kRankPer = 4, kRankPhases = 64;
constexpr uint32_t kRankGroups = kRankKeys / kRankPer;        // 8 groups of 4 keys
constexpr uint32_t kRankThreads = kRankGroups * kRankPhases;  // 512: a group is two warps
constexpr uint32_t kRankEarly = 512;                           // keys copied before the count is known

__global__ void __launch_bounds__(kRankThreads)
    rank_sort_kernel(const unsigned long long *__restrict__ keys, const unsigned long long *num, uint64_t cap,
                     uint32_t shift, ac_match *__restrict__ out, unsigned long long *num_out, const uint32_t *err) {
    extern __shared__ __align__(16) unsigned long long sk[];  // pairs(cap) * 2 keys
    __shared__ uint32_t part[kRankGroups][2][kRankPer];      // per group: each warp's counts
    kern::pdl_release();  // the next call's zeroing may start; it waits for this launch before writing
    kern::pdl_wait();     // the keys, the counter and the error word of the launch before
    const uint32_t base = smem_addr(sk);
    const bool aligned = ((uintptr_t)keys & 15) == 0;
    // the first keys' copies go out with the count's read (copies past the
    // count read unused entries of the buffer, never past its capacity)
    const uint32_t early = (uint32_t)(cap < kRankEarly ? cap : kRankEarly) / 2;  // pairs
    if (aligned && blockIdx.x * kRankKeys < cap)
        for (uint32_t t = threadIdx.x; t < early; t += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(base + 16 * t), "l"(keys + 2 * t)
                         : "memory");
    const unsigned long long M = *num;  // num_out may be num: read before anything is written
    const bool failed = err && *err;
    if (blockIdx.x == 0 && threadIdx.x == 0 && num_out) *num_out = failed ? ~0ull : M;
    const uint32_t m = (uint32_t)(M < cap ? M : cap);
    const uint32_t kb = blockIdx.x * kRankKeys;
    if (failed || kb >= m) {  // uniform across the CTA
        asm volatile("cp.async.wait_all;" ::: "memory");  // no copy outlives the CTA
        return;
    }
    const uint32_t pairs = (m + 1) / 2;
    if (aligned) {
        for (uint32_t t = early + threadIdx.x; t < m / 2; t += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(base + 16 * t), "l"(keys + 2 * t)
                         : "memory");
    } else {  // keys only 8-byte aligned
        for (uint32_t t = threadIdx.x; t < m / 2 * 2; t += blockDim.x) sk[t] = keys[t];
    }
    const unsigned long long last = (m & 1) && threadIdx.x == 0 ? keys[m - 1] : 0ull;
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // an odd count's last pair is the last key and the all-ones pad (never
    // below a key), written once every copy has landed
    if ((m & 1) && threadIdx.x == 0) {
        sk[m - 1] = last;
        sk[m] = ~0ull;
    }
    __syncthreads();
    const uint32_t ph = threadIdx.x % kRankPhases, grp = threadIdx.x / kRankPhases;
    unsigned long long ki[kRankPer];
#pragma unroll
    for (uint32_t r = 0; r < kRankPer; ++r) {
        const uint32_t i = kb + grp * kRankPer + r;
        ki[r] = i < m ? sk[i] : ~0ull;
    }
    const uint4 *sk4 = reinterpret_cast<const uint4 *>(sk);
    uint32_t below[kRankPer] = {0, 0, 0, 0};
#pragma unroll 2
    for (uint32_t j = ph; j < pairs; j += kRankPhases) {
        const uint4 v = sk4[j];  // keys 2j and 2j + 1
        const unsigned long long x = ((unsigned long long)v.y << 32) | v.x;
        const unsigned long long y = ((unsigned long long)v.w << 32) | v.z;
#pragma unroll
        for (uint32_t r = 0; r < kRankPer; ++r) below[r] += (x < ki[r] ? 1u : 0u) + (y < ki[r] ? 1u : 0u);
    }
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (uint32_t r = 0; r < kRankPer; ++r) {
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) below[r] += __shfl_xor_sync(kFull, below[r], o);
        if (lane == 0) part[grp][(threadIdx.x / 32) & 1][r] = below[r];
    }
    __syncthreads();
    if (threadIdx.x < kRankKeys) {
        const uint32_t g = threadIdx.x / kRankPer, r = threadIdx.x % kRankPer;
        const uint32_t i = kb + threadIdx.x;
        if (i < m) {
            const unsigned long long k = sk[i];
            ac_match rec;
            rec.pos = (uint32_t)(k >> shift);
            rec.pattern_id = (uint32_t)(k & ((1ull << shift) - 1ull));
            out[part[g][0][r] + part[g][1][r]] = rec;
        }
    }
}
}  // namespace

// The rank sort's shared-memory attribute, set once per process.
static cudaError_t small_sort_attr() {
    static std::once_flag once;
    static cudaError_t attr = cudaSuccess;
    std::call_once(once, [] {
        attr = cudaFuncSetAttribute(rank_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)((kSmallSortMax / 2 + 1) * 16));
    });
    return attr;
}

void prime_scan_state() {
    (void)encoder();
    (void)small_sort_attr();
}

int launch_small_sort(const unsigned long long *keys, const unsigned long long *num, uint64_t cap, uint32_t shift,
                      ac_match *out, unsigned long long *num_out, const uint32_t *err, cudaStream_t stream,
                      bool overlap) {
    if (cap > kSmallSortMax) return set_error(AC_EINVAL, "small sort: capacity above %llu",
                                              (unsigned long long)kSmallSortMax);
    const int smem = (int)(((cap + 1) / 2 + 1) * 16);
    const cudaError_t attr = small_sort_attr();
    if (attr != cudaSuccess) return set_error(AC_ECUDA, "small sort: %s", cudaGetErrorString(attr));
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, (cap + kRankKeys - 1) / kRankKeys);
    cudaError_t e = launch_overlapped(rank_sort_kernel, dim3(grid), dim3(kRankThreads), (size_t)smem, stream, overlap,
                                      keys, num, cap, shift, out, num_out, err);
    return e == cudaSuccess ? AC_OK : set_error(AC_ECUDA, "small sort: %s", cudaGetErrorString(e));
}

int sort_keys(unsigned long long *keys, unsigned long long *keys_alt, uint64_t count, int begin_bit, int end_bit,
              void *temp, size_t *temp_bytes, cudaStream_t stream, unsigned long long **sorted) {
    if (count > 0x7fffffffull) return set_error(AC_ERANGE, "sort: too many matches");
    cub::DoubleBuffer<unsigned long long> db(keys, keys_alt);
    cudaError_t e = cub::DeviceRadixSort::SortKeys(temp, *temp_bytes, db, (int)count, begin_bit, end_bit, stream);
    if (e != cudaSuccess) return set_error(AC_ECUDA, "sort: %s", cudaGetErrorString(e));
    if (sorted) *sorted = db.Current();
    return AC_OK;
}

}  // namespace acgb
