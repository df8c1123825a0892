// ac_scan_batch: many texts, each against one of several resident automata,
// in one persistent launch.
//
// Layout: the texts are copied into one device arena of whole rows (every
// text starts on a row boundary; its last row is padded), grouped by
// automaton, each group padded to a whole number of tiles so a CTA's tile
// uses one automaton's table. One 2-D tensor map covers the arena; a tile
// list names the machine (automaton subset) and first row of every tile; a
// chain finds its text by binary search over the items. Match keys carry the
// arena position of the match, so one sort orders every text's matches, and
// the sorted keys split per text by binary search.
//
// Repeated batches: with AC_BATCH_GRAPH the plan (layout, buffers, chosen
// configuration) is kept, keyed by the automata, text pointers, lengths and
// formats, and the whole device sequence (text copies, scan, sort, record
// conversion, copies back) is captured once in a CUDA graph and replayed.
// The first call of such a plan autotunes the row length and the CTA shape
// by timing candidates on the real batch.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>

#include <cub/device/device_radix_sort.cuh>

#include "ac_internal.h"

namespace acgb {
namespace {

uint32_t value_bits(uint64_t x) {
    uint32_t b = 1;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

// sorted keys -> (position within the text, pattern id)
__global__ void batch_records_kernel(const unsigned long long *__restrict__ keys, const unsigned long long *num,
                                     uint64_t cap, uint32_t shift, const BatchItemDev *__restrict__ items,
                                     uint32_t ni, ac_match *__restrict__ out) {
    const unsigned long long M = *num;
    const uint64_t m = M < cap ? M : cap;
    const unsigned long long mask = (1ull << shift) - 1ull;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        const uint64_t v = k >> shift;
        uint32_t lo = 0, hi = ni;  // first item whose vbase > v
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (items[mid].vbase <= v) lo = mid + 1;
            else hi = mid;
        }
        const uint64_t base = lo ? items[lo - 1].vbase : 0;
        ac_match r;
        r.pos = (uint32_t)(v - base);
        r.pattern_id = (uint32_t)(k & mask);
        out[i] = r;
    }
}

// off[i] = index of the first sorted key of item i; off[ni] = min(M, cap)
__global__ void batch_offsets_kernel(const unsigned long long *__restrict__ keys, const unsigned long long *num,
                                     uint64_t cap, uint32_t shift, const BatchItemDev *__restrict__ items,
                                     uint32_t ni, unsigned long long *__restrict__ off) {
    const unsigned long long M = *num;
    const uint64_t m = M < cap ? M : cap;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= ni; i += gridDim.x * blockDim.x) {
        if (i == ni) {
            off[i] = m;
            continue;
        }
        const unsigned long long first = (unsigned long long)items[i].vbase << shift;
        uint64_t lo = 0, hi = m;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (keys[mid] < first) lo = mid + 1;
            else hi = mid;
        }
        off[i] = lo;
    }
}

struct Plan {
    int device = 0, fmt = AC_U8, mem = AC_HOST;
    cudaStream_t pool_stream = nullptr;  // transient plans: buffers from the stream-ordered pool
    bool pooled = false;
    uint32_t flags = 0;
    std::vector<uint32_t> caller;        // plan order -> caller's item index
    std::vector<const uint8_t *> src;    // plan order -> text
    std::vector<uint64_t> nbytes;        // plan order
    std::vector<uint32_t> npat;          // plan order -> patterns of its automaton
    std::vector<BatchItemDev> items;
    std::vector<BatchTileDev> tiles;
    std::vector<SubsetDev> machines;
    uint64_t rows = 0, total_counts = 0, cap = 0;
    uint32_t row_bytes = 0, key_shift = 1, max_states = 0, sigma = 0;
    bool acgt = false;
    uint8_t sym[256];
    int placement = AC_PLACE_AUTO;
    uint32_t smem_cap = 0;
    ac_scan_config cfg{};
    // device buffers
    uint8_t *d_arena = nullptr;
    BatchItemDev *d_items = nullptr;
    BatchTileDev *d_tiles = nullptr;
    SubsetDev *d_machines = nullptr;
    unsigned long long *d_num = nullptr;  // [0] count, [1] error word
    unsigned long long *d_keys = nullptr, *d_alt = nullptr, *d_counts = nullptr, *d_off = nullptr;
    ac_match *d_rec = nullptr;
    void *d_sort = nullptr;
    size_t sort_bytes = 0;
    // pinned host buffers (graph plans)
    uint8_t *h_stage = nullptr;
    ac_match *h_rec = nullptr;
    unsigned long long *h_off = nullptr, *h_counts = nullptr, *h_num = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t arena_bytes() const { return rows * row_bytes; }
};

void free_plan_buffers(Plan &P) {
    void *dev[] = {P.d_arena, P.d_items, P.d_tiles, P.d_machines, P.d_num, P.d_keys, P.d_alt,
                   P.d_counts, P.d_off, P.d_rec, P.d_sort};
    for (void *p : dev)
        if (p) {
            if (P.pooled) dev_free(p, P.pool_stream);
            else cudaFree(p);
        }
    void *host[] = {P.h_stage, P.h_rec, P.h_off, P.h_counts, P.h_num};
    for (void *p : host)
        if (p) cudaFreeHost(p);
    if (P.exec) cudaGraphExecDestroy(P.exec);
    P.d_arena = nullptr;
    P.d_items = nullptr;
    P.d_tiles = nullptr;
    P.d_machines = nullptr;
    P.d_num = P.d_keys = P.d_alt = P.d_counts = P.d_off = nullptr;
    P.d_rec = nullptr;
    P.d_sort = nullptr;
    P.h_stage = nullptr;
    P.h_rec = nullptr;
    P.h_off = P.h_counts = P.h_num = nullptr;
    P.exec = nullptr;
}

// Lay out the items idx[] (all of one alphabet class) for row length
// row_bytes and CTA shape cfg.
int layout(const ac_automaton *const *as, const ac_batch_item *items, const std::vector<uint32_t> &idx,
           uint32_t row_bytes, const ac_scan_config &cfg, uint32_t flags, Plan &P) {
    P.row_bytes = row_bytes;
    P.cfg = cfg;
    P.cfg.row_len = 0;
    const uint32_t R = cfg.threads * cfg.chains;  // rows per tile
    const uint32_t spb = P.fmt == AC_U8 ? 1 : 4;
    P.caller.clear();
    P.src.clear();
    P.nbytes.clear();
    P.npat.clear();
    P.items.clear();
    P.tiles.clear();
    P.machines.clear();
    // stable order by automaton
    std::vector<uint32_t> order(idx);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return items[x].automaton < items[y].automaton; });
    uint64_t row = 0, counts = 0;
    uint32_t maxP = 1;
    size_t g = 0;
    while (g < order.size()) {
        const uint32_t aidx = items[order[g]].automaton;
        const ac_automaton *a = as[aidx];
        const uint32_t mbase = (uint32_t)P.machines.size();
        for (auto &d : a->h_desc) P.machines.push_back(d);
        maxP = std::max(maxP, a->P);
        const uint64_t group_row0 = row;
        size_t e = g;
        for (; e < order.size() && items[order[e]].automaton == aidx; ++e) {
            const ac_batch_item &it = items[order[e]];
            const uint64_t nb = P.fmt == AC_U8 ? it.n : (it.n + 3) / 4;
            BatchItemDev d{};
            d.row_begin = row;
            d.rows = (nb + row_bytes - 1) / row_bytes;
            d.nsym = it.n;
            d.vbase = row * row_bytes * spb;
            d.cbase = counts;
            P.items.push_back(d);
            P.caller.push_back(order[e]);
            P.src.push_back(it.text);
            P.nbytes.push_back(nb);
            P.npat.push_back(a->P);
            row += d.rows;
            if (!(flags & AC_BATCH_NO_COUNTS)) counts += a->P;
        }
        // pad the group to whole tiles and list its tiles (subsets fastest)
        row = (row + R - 1) / R * R;
        for (uint64_t r0 = group_row0; r0 < row; r0 += R)
            for (uint32_t k = 0; k < a->K; ++k) P.tiles.push_back(BatchTileDev{mbase + k, 0, r0});
        g = e;
    }
    P.rows = row;
    P.total_counts = counts;
    P.key_shift = value_bits(maxP - 1);
    P.max_states = 0;
    for (auto &m : P.machines) P.max_states = std::max(P.max_states, m.states);
    const uint64_t top = P.rows * P.row_bytes * spb;
    if (P.rows >= (1ull << 31) || P.key_shift + value_bits(top) > 64)
        return set_error(AC_ERANGE, "ac_scan_batch: batch too large for one launch");
    return AC_OK;
}

uint32_t default_row_bytes(uint64_t total_bytes, uint32_t max_warm_bytes, const ac_scan_config &cfg, int device) {
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const uint64_t chains = (uint64_t)sms * cfg.threads * cfg.chains;
    uint64_t L = (total_bytes + 2 * chains - 1) / (2 * chains);  // about two rows per chain
    L = std::max<uint64_t>(L, std::max<uint64_t>(256, 8ull * max_warm_bytes));
    L = std::min<uint64_t>(L, 1u << 22);
    return (uint32_t)((L + kStageBytes - 1) / kStageBytes * kStageBytes);
}

int alloc_dev(void **p, size_t bytes, const Plan &P) {
    if (P.pooled) {
        *p = dev_alloc(bytes ? bytes : 16, P.pool_stream);
        return *p ? AC_OK : set_error(AC_ENOMEM, "ac_scan_batch: device memory (%zu bytes)", bytes);
    }
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(e == cudaErrorMemoryAllocation ? AC_ENOMEM : AC_ECUDA, "ac_scan_batch: %s",
                         cudaGetErrorString(e));
    }
    return AC_OK;
}

#define BCK(call, what)                                                                                   \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) {                                                                          \
            cudaGetLastError();                                                                           \
            return set_error(e_ == cudaErrorMemoryAllocation ? AC_ENOMEM : AC_ECUDA, "%s: %s", what,     \
                             cudaGetErrorString(e_));                                                     \
        }                                                                                                 \
    } while (0)

// (Re)allocate the device buffers of a plan for its layout and capacity.
int alloc_plan(Plan &P, uint64_t cap) {
    P.cap = cap;
    const uint32_t ni = (uint32_t)P.items.size();
    int rc;
    if ((rc = alloc_dev((void **)&P.d_arena, P.arena_bytes(), P))) return rc;
    if ((rc = alloc_dev((void **)&P.d_items, ni * sizeof(BatchItemDev), P))) return rc;
    if ((rc = alloc_dev((void **)&P.d_tiles, P.tiles.size() * sizeof(BatchTileDev), P))) return rc;
    if ((rc = alloc_dev((void **)&P.d_machines, P.machines.size() * sizeof(SubsetDev), P))) return rc;
    if ((rc = alloc_dev((void **)&P.d_num, 16, P))) return rc;
    if ((rc = alloc_dev((void **)&P.d_keys, cap * 8, P))) return rc;
    if ((rc = alloc_dev((void **)&P.d_alt, cap * 8, P))) return rc;
    if ((rc = alloc_dev((void **)&P.d_rec, cap * 8, P))) return rc;
    if ((rc = alloc_dev((void **)&P.d_off, (ni + 1) * 8, P))) return rc;
    if (P.total_counts && (rc = alloc_dev((void **)&P.d_counts, P.total_counts * 8, P))) return rc;
    const int end_bit = (int)std::min<uint32_t>(64, P.key_shift + value_bits(P.rows * P.row_bytes * 4));
    P.sort_bytes = 0;
    cub::DoubleBuffer<unsigned long long> db(P.d_keys, P.d_alt);
    BCK(cub::DeviceRadixSort::SortKeys(nullptr, P.sort_bytes, db, (int)cap, 0, end_bit), "ac_scan_batch: sort size");
    if ((rc = alloc_dev(&P.d_sort, P.sort_bytes, P))) return rc;
    if (P.pooled) {
        cudaStream_t s = P.pool_stream;
        BCK(cudaMemcpyAsync(P.d_items, P.items.data(), ni * sizeof(BatchItemDev), cudaMemcpyHostToDevice, s),
            "ac_scan_batch");
        BCK(cudaMemcpyAsync(P.d_tiles, P.tiles.data(), P.tiles.size() * sizeof(BatchTileDev), cudaMemcpyHostToDevice,
                            s),
            "ac_scan_batch");
        BCK(cudaMemcpyAsync(P.d_machines, P.machines.data(), P.machines.size() * sizeof(SubsetDev),
                            cudaMemcpyHostToDevice, s),
            "ac_scan_batch");
        return AC_OK;
    }
    BCK(cudaMemcpy(P.d_items, P.items.data(), ni * sizeof(BatchItemDev), cudaMemcpyHostToDevice), "ac_scan_batch");
    BCK(cudaMemcpy(P.d_tiles, P.tiles.data(), P.tiles.size() * sizeof(BatchTileDev), cudaMemcpyHostToDevice),
        "ac_scan_batch");
    BCK(cudaMemcpy(P.d_machines, P.machines.data(), P.machines.size() * sizeof(SubsetDev), cudaMemcpyHostToDevice),
        "ac_scan_batch");
    return AC_OK;
}

BatchLaunch launch_of(const Plan &P) {
    BatchLaunch b{};
    b.arena = P.d_arena;
    b.rows = P.rows;
    b.row_bytes = P.row_bytes;
    b.fmt = P.fmt;
    b.items = P.d_items;
    b.num_items = (uint32_t)P.items.size();
    b.tiles = P.d_tiles;
    b.num_tiles = P.tiles.size();
    b.machines = P.d_machines;
    b.max_states = P.max_states;
    b.sigma = P.sigma;
    b.sym_of_byte = P.sym;
    b.acgt = P.acgt;
    b.key_shift = P.key_shift;
    b.placement = P.placement;
    b.smem_cap_bytes = P.smem_cap;
    b.device = P.device;
    b.cfg = P.cfg;
    b.track_flags = 1;  // a batch's machines each hold a whole pattern set
    return b;
}

// Copy the texts into the arena (from the pinned stage for graph plans of host texts).
int copy_texts(Plan &P, cudaStream_t s, bool from_stage) {
    uint64_t off = 0;
    for (size_t i = 0; i < P.items.size(); ++i) {
        if (!P.nbytes[i]) continue;
        uint8_t *dst = P.d_arena + P.items[i].row_begin * P.row_bytes;
        const uint8_t *src = from_stage ? P.h_stage + off : P.src[i];
        const cudaMemcpyKind kind = (P.mem == AC_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        BCK(cudaMemcpyAsync(dst, src, P.nbytes[i], kind, s), "ac_scan_batch: text copy");
        off += P.nbytes[i];
    }
    return AC_OK;
}

// Everything after the text copies: clear, scan, sort cap keys, records,
// offsets. Capturable (no host synchronisation).
int device_sequence(Plan &P, cudaStream_t s) {
    BCK(cudaMemsetAsync(P.d_num, 0, 16, s), "ac_scan_batch: memset");
    if (P.d_counts) BCK(cudaMemsetAsync(P.d_counts, 0, P.total_counts * 8, s), "ac_scan_batch: memset");
    ScanOut o{P.d_keys, P.cap, P.d_num, P.d_counts, (uint32_t *)(P.d_num + 1)};
    int rc = launch_scan_batch(launch_of(P), o, s);
    if (rc) return rc;
    rc = launch_pad_keys(P.d_keys, P.d_num, P.cap, s);
    if (rc) return rc;
    const int end_bit = (int)std::min<uint32_t>(64, P.key_shift + value_bits(P.rows * P.row_bytes * 4));
    unsigned long long *sorted = nullptr;
    size_t tb = P.sort_bytes;
    rc = sort_keys(P.d_keys, P.d_alt, P.cap, 0, end_bit, P.d_sort, &tb, s, &sorted);
    if (rc) return rc;
    const uint32_t ni = (uint32_t)P.items.size();
    uint64_t blocks = std::min<uint64_t>(2048, (P.cap + 255) / 256);
    batch_records_kernel<<<(unsigned)std::max<uint64_t>(1, blocks), 256, 0, s>>>(sorted, P.d_num, P.cap, P.key_shift,
                                                                                  P.d_items, ni, P.d_rec);
    batch_offsets_kernel<<<(ni + 256) / 256, 256, 0, s>>>(sorted, P.d_num, P.cap, P.key_shift, P.d_items, ni,
                                                          P.d_off);
    BCK(cudaGetLastError(), "ac_scan_batch: records");
    return AC_OK;
}

// Results from host copies of records, offsets, counts.
int split_results(const Plan &P, const ac_match *rec, const unsigned long long *off, const unsigned long long *counts,
                  ac_result *outs) {
    for (size_t j = 0; j < P.items.size(); ++j) {
        ac_result &r = outs[P.caller[j]];
        r.num_patterns = P.npat[j];
        const uint64_t b = off[j], e = off[j + 1];
        r.num_matches = e - b;
        if (e > b) {
            r.matches = (ac_match *)malloc((e - b) * sizeof(ac_match));
            if (!r.matches) return set_error(AC_ENOMEM, "ac_scan_batch: host results");
            memcpy(r.matches, rec + b, (e - b) * sizeof(ac_match));
        }
        if (counts) {
            r.counts = (uint64_t *)malloc((size_t)P.npat[j] * 8);
            if (!r.counts) return set_error(AC_ENOMEM, "ac_scan_batch: host counts");
            memcpy(r.counts, counts + P.items[j].cbase, (size_t)P.npat[j] * 8);
        }
    }
    return AC_OK;
}

// One synchronous run of a plan (buffers allocated, texts not yet copied).
int run_once(Plan &P, cudaStream_t s, ac_result *outs, uint64_t *M_out) {
    int rc = copy_texts(P, s, false);
    if (rc) return rc;
    rc = device_sequence(P, s);
    if (rc) return rc;
    unsigned long long h[2];
    BCK(cudaMemcpyAsync(h, P.d_num, 16, cudaMemcpyDeviceToHost, s), "ac_scan_batch: count");
    BCK(cudaStreamSynchronize(s), "ac_scan_batch: scan");
    if ((uint32_t)h[1]) return set_error(AC_ETIMEDOUT, "ac_scan_batch: a device-side wait ran out");
    *M_out = h[0];
    if (h[0] > P.cap) return AC_OK;  // caller grows cap and retries
    const uint32_t ni = (uint32_t)P.items.size();
    std::vector<ac_match> rec(h[0]);
    std::vector<unsigned long long> off(ni + 1);
    std::vector<unsigned long long> counts(P.total_counts);
    if (h[0]) BCK(cudaMemcpyAsync(rec.data(), P.d_rec, h[0] * 8, cudaMemcpyDeviceToHost, s), "ac_scan_batch");
    BCK(cudaMemcpyAsync(off.data(), P.d_off, (ni + 1) * 8, cudaMemcpyDeviceToHost, s), "ac_scan_batch");
    if (P.total_counts)
        BCK(cudaMemcpyAsync(counts.data(), P.d_counts, P.total_counts * 8, cudaMemcpyDeviceToHost, s),
            "ac_scan_batch");
    BCK(cudaStreamSynchronize(s), "ac_scan_batch: results");
    return split_results(P, rec.data(), off.data(), P.total_counts ? counts.data() : nullptr, outs);
}

// ---------------------------------------------------------------- graph plans
struct PlanKey {
    std::vector<uintptr_t> v;
    bool operator<(const PlanKey &o) const { return v < o.v; }
};

std::mutex g_plan_mu;
std::map<PlanKey, std::unique_ptr<Plan>> g_plans;  // at most kMaxPlans kept
constexpr size_t kMaxPlans = 2;

// Time the scan of a laid-out plan (texts already in the arena).
float time_scan(Plan &P, cudaStream_t s) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    ScanOut o{P.d_keys, P.cap, P.d_num, nullptr, (uint32_t *)(P.d_num + 1)};
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaMemsetAsync(P.d_num, 0, 16, s);
        cudaEventRecord(e0, s);
        if (launch_scan_batch(launch_of(P), o, s) != AC_OK) break;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// ------------------------------------------------------------ texts as one text per automaton
// Byte texts whose alphabet leaves a byte free are scanned one automaton at a
// time as one text: the automaton's texts are laid end to end in one device
// buffer, each starting on a 16-byte boundary behind at least one byte outside
// the alphabet. That byte sends the walk back to the root (Section II.A: no
// pattern contains it), so every text is walked exactly as if alone, and the
// buffer goes through the single-text path (its automatic kernel choice for
// the buffer's length). The sorted matches split per text by position; a
// text's counts are the histogram of its matches.

constexpr uint64_t kSegmentMaxBytes = 1ull << 31;  // bytes of texts in one segment (positions stay 32-bit)
constexpr uint64_t kGatherChunk = 256u << 10;     // bytes one CTA of the gather copies

struct GatherChunk {
    const uint8_t *src;  // null: fill with the separator byte
    uint8_t *dst;
    uint64_t len;
};

// Device texts into their places in the segment buffers and the separator
// bytes around them, one chunk per CTA.
__global__ void gather_kernel(const GatherChunk *__restrict__ chunks, uint8_t sep) {
    const GatherChunk c = chunks[blockIdx.x];
    uint8_t *d = c.dst;
    if (!c.src) {
        for (uint64_t i = threadIdx.x; i < c.len; i += blockDim.x) d[i] = sep;
    } else if ((((uintptr_t)c.src | (uintptr_t)d) & 15) == 0) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(c.src);
        uint4 *d4 = reinterpret_cast<uint4 *>(d);
        const uint64_t n4 = c.len / 16;
        for (uint64_t i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = __ldg(s4 + i);
        for (uint64_t i = n4 * 16 + threadIdx.x; i < c.len; i += blockDim.x) d[i] = c.src[i];
    } else {
        for (uint64_t i = threadIdx.x; i < c.len; i += blockDim.x) d[i] = c.src[i];
    }
}

// The byte of `a`'s symbol map that lies outside its alphabet, or -1.
int separator_byte(const ac_automaton *a) {
    for (int b = 0; b < 256; ++b)
        if (a->sym_of_byte[b] >= a->sigma) return b;
    return -1;
}

struct Segment {
    const ac_automaton *a = nullptr;
    std::vector<uint32_t> item;   // caller's item indices, in layout order
    std::vector<uint64_t> off;    // byte offset of each text in the buffer
    uint64_t len = 0;             // bytes from the buffer start to the last text's end
    uint64_t alloc = 0;
    uint8_t *buf = nullptr;
    unsigned long long *keys = nullptr;
    uint64_t cap = 0;
    EmitEntry *q = nullptr;  // lean kernel's emission queue
    uint64_t q_cap = 0;
};

int scan_segments(const ac_automaton *const *as, const ac_batch_item *items, const std::vector<uint32_t> &idx,
                  int mem, uint32_t flags, uint8_t sep, cudaStream_t s, ac_result *outs) {
    struct Pool {  // stream-ordered scratch, released when the call ends
        cudaStream_t s;
        std::vector<void *> ptrs;
        void *get(size_t bytes) {
            void *p = dev_alloc(bytes, s);
            if (p) ptrs.push_back(p);
            return p;
        }
        ~Pool() {
            for (void *p : ptrs) dev_free(p, s);
        }
    } pool{s, {}};
    // segments: automata in index order, the caller's order within one
    std::vector<uint32_t> order(idx);
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return items[x].automaton < items[y].automaton; });
    std::vector<Segment> segs;
    for (uint32_t i : order) {
        const ac_automaton *a = as[items[i].automaton];
        const uint64_t n = items[i].n;
        const uint64_t at = segs.empty() || segs.back().a != a ? 0 : (segs.back().len + 1 + 15) / 16 * 16;
        if (segs.empty() || segs.back().a != a || at + n > kSegmentMaxBytes) {
            segs.emplace_back();
            segs.back().a = a;
            segs.back().item.push_back(i);
            segs.back().off.push_back(0);
            segs.back().len = n;
        } else {
            segs.back().item.push_back(i);
            segs.back().off.push_back(at);
            segs.back().len = at + n;
        }
    }
    const size_t G = segs.size();
    // buffers; the texts (host texts copied one by one, device texts by the
    // gather) and the separator bytes between and after them (the gather)
    std::vector<GatherChunk> chunks;
    for (size_t g = 0; g < G; ++g) {
        Segment &sg = segs[g];
        sg.alloc = std::max<uint64_t>((sg.len + 15) / 16 * 16, kStageBytes);
        sg.buf = (uint8_t *)pool.get(sg.alloc);
        if (!sg.buf) return set_error(AC_ENOMEM, "ac_scan_batch: text buffer of %llu bytes", (unsigned long long)sg.alloc);
        for (size_t k = 0; k < sg.item.size(); ++k) {
            const ac_batch_item &it = items[sg.item[k]];
            if (mem == AC_HOST) {
                BCK(cudaMemcpyAsync(sg.buf + sg.off[k], it.text, it.n, cudaMemcpyHostToDevice, s),
                    "ac_scan_batch: text copy");
            } else {
                for (uint64_t c0 = 0; c0 < it.n; c0 += kGatherChunk)
                    chunks.push_back(GatherChunk{it.text + c0, sg.buf + sg.off[k] + c0, std::min(kGatherChunk, it.n - c0)});
            }
            const uint64_t end = sg.off[k] + it.n;
            const uint64_t next = k + 1 < sg.item.size() ? sg.off[k + 1] : sg.alloc;
            if (next > end) chunks.push_back(GatherChunk{nullptr, sg.buf + end, next - end});
        }
    }
    if (!chunks.empty()) {
        GatherChunk *d_chunks = (GatherChunk *)pool.get(chunks.size() * sizeof(GatherChunk));
        if (!d_chunks) return set_error(AC_ENOMEM, "ac_scan_batch: gather list");
        BCK(cudaMemcpyAsync(d_chunks, chunks.data(), chunks.size() * sizeof(GatherChunk), cudaMemcpyHostToDevice, s),
            "ac_scan_batch: gather list");
        for (uint64_t c0 = 0; c0 < chunks.size(); c0 += 65535) {  // at most 65,535 CTAs a launch here
            const unsigned grid = (unsigned)std::min<uint64_t>(65535, chunks.size() - c0);
            gather_kernel<<<grid, 256, 0, s>>>(d_chunks + c0, sep);
        }
        BCK(cudaGetLastError(), "ac_scan_batch: gather");
    }
    // counters: [2g] matches of segment g, [2g + 1] its error word
    unsigned long long *d_ctr = (unsigned long long *)pool.get(G * 16);
    if (!d_ctr) return set_error(AC_ENOMEM, "ac_scan_batch: counters");
    std::vector<unsigned long long> h_ctr(2 * G);
    auto scan_all = [&](const std::vector<size_t> &which) -> int {
        for (size_t g : which) {
            BCK(cudaMemsetAsync(d_ctr + 2 * g, 0, 16, s), "ac_scan_batch: counters");
            Segment &sg = segs[g];
            ac_scan_config cfg;
            default_config(sg.a, sg.len, AC_U8, &cfg);
            ScanText t{sg.buf, sg.len, AC_U8, sg.alloc};
            ScanOut o{sg.keys, sg.cap, d_ctr + 2 * g, nullptr, (uint32_t *)(d_ctr + 2 * g + 1)};
            if (cfg.kernel == AC_KERNEL_LEAN && sg.a->machine == AC_MACHINE_DFA) {
                // the lean kernel's emission queue (none: stages with matches are walked again in place)
                if (!sg.q) {
                    sg.q_cap = emit_queue_cap(sg.len, AC_U8);
                    sg.q = (EmitEntry *)pool.get(sg.q_cap * sizeof(EmitEntry));
                }
                if (sg.q) {
                    o.q = sg.q;
                    o.q_cap = sg.q_cap;
                }
            }
            const int rc = launch_scan(sg.a, t, o, cfg, s);
            if (rc) return rc;
        }
        BCK(cudaMemcpyAsync(h_ctr.data(), d_ctr, G * 16, cudaMemcpyDeviceToHost, s), "ac_scan_batch: counters");
        BCK(cudaStreamSynchronize(s), "ac_scan_batch: scan");
        for (size_t g : which)
            if ((uint32_t)h_ctr[2 * g + 1]) return set_error(AC_ETIMEDOUT, "ac_scan_batch: a device-side wait ran out");
        return AC_OK;
    };
    std::vector<size_t> all(G);
    std::iota(all.begin(), all.end(), 0);
    for (Segment &sg : segs) {
        sg.cap = std::min<uint64_t>(sg.len / 256 + 4096, 1ull << 26);
        sg.keys = (unsigned long long *)pool.get(sg.cap * 8);
        if (!sg.keys) return set_error(AC_ENOMEM, "ac_scan_batch: match keys");
    }
    int rc = scan_all(all);
    if (rc) return rc;
    std::vector<size_t> over;
    for (size_t g = 0; g < G; ++g)
        if (h_ctr[2 * g] > segs[g].cap) {  // more matches than room: scan again with room for all
            segs[g].cap = h_ctr[2 * g];
            segs[g].keys = (unsigned long long *)pool.get(segs[g].cap * 8);
            if (!segs[g].keys) return set_error(AC_ENOMEM, "ac_scan_batch: match keys");
            over.push_back(g);
        }
    if (!over.empty() && (rc = scan_all(over))) return rc;
    // sort each segment's keys into records, bring them back
    std::vector<std::vector<ac_match>> rec(G);
    for (size_t g = 0; g < G; ++g) {
        Segment &sg = segs[g];
        const uint64_t M = h_ctr[2 * g];
        if (!M) continue;
        ac_match *d_rec = (ac_match *)pool.get(M * sizeof(ac_match));
        if (!d_rec) return set_error(AC_ENOMEM, "ac_scan_batch: records");
        const uint32_t shift = (uint32_t)key_shift_for(sg.a);
        if (M <= kSmallSortMax) {
            rc = launch_small_sort(sg.keys, d_ctr + 2 * g, M, shift, d_rec, nullptr, nullptr, s);
        } else {
            unsigned long long *alt = (unsigned long long *)pool.get(M * 8);
            if (!alt) return set_error(AC_ENOMEM, "ac_scan_batch: sort buffer");
            const int end_bit = (int)std::min<uint32_t>(64, shift + value_bits(sg.len ? sg.len - 1 : 0));
            size_t tb = 0;
            rc = sort_keys(sg.keys, alt, M, sort_begin_bit(sg.a), end_bit, nullptr, &tb, s, nullptr);
            void *temp = rc ? nullptr : pool.get(tb);
            if (!rc && !temp) return set_error(AC_ENOMEM, "ac_scan_batch: sort scratch");
            unsigned long long *sorted = nullptr;
            if (!rc) rc = sort_keys(sg.keys, alt, M, sort_begin_bit(sg.a), end_bit, temp, &tb, s, &sorted);
            if (!rc) rc = launch_keys_to_matches(sorted, d_ctr + 2 * g, M, shift, d_rec, nullptr, nullptr, s);
        }
        if (rc) return rc;
        rec[g].resize(M);
        BCK(cudaMemcpyAsync(rec[g].data(), d_rec, M * sizeof(ac_match), cudaMemcpyDeviceToHost, s),
            "ac_scan_batch: records");
    }
    BCK(cudaStreamSynchronize(s), "ac_scan_batch: sort");
    // split per text (records are sorted by position; texts are in position order)
    const bool counts = !(flags & AC_BATCH_NO_COUNTS);
    for (size_t g = 0; g < G; ++g) {
        const Segment &sg = segs[g];
        size_t r = 0;
        for (size_t k = 0; k < sg.item.size(); ++k) {
            ac_result &o = outs[sg.item[k]];
            o.num_patterns = sg.a->P;
            const uint64_t lo = sg.off[k], hi = sg.off[k] + items[sg.item[k]].n;
            while (r < rec[g].size() && rec[g][r].pos < lo) ++r;  // none: separators hold no match
            size_t e = r;
            while (e < rec[g].size() && rec[g][e].pos < hi) ++e;
            o.num_matches = e - r;
            if (e > r) {
                o.matches = (ac_match *)malloc((e - r) * sizeof(ac_match));
                if (!o.matches) return set_error(AC_ENOMEM, "ac_scan_batch: host results");
                for (size_t q = r; q < e; ++q) o.matches[q - r] = ac_match{(uint32_t)(rec[g][q].pos - lo), rec[g][q].pattern_id};
            }
            if (counts) {
                o.counts = (uint64_t *)calloc(sg.a->P ? sg.a->P : 1, 8);
                if (!o.counts) return set_error(AC_ENOMEM, "ac_scan_batch: host counts");
                for (size_t q = r; q < e; ++q) o.counts[rec[g][q].pattern_id]++;
            }
            r = e;
        }
    }
    return AC_OK;
}

}  // namespace
}  // namespace acgb

using namespace acgb;

extern "C" int ac_scan_batch(const ac_automaton *const *as, uint32_t na, const ac_batch_item *items, uint32_t ni,
                             int mem, uint32_t flags, void *stream, ac_result *outs) {
    NvtxRange nvtx_range("ac_scan_batch");
    if (!as || !na || (!items && ni) || (!outs && ni)) return set_error(AC_EINVAL, "ac_scan_batch: NULL argument");
    if (mem != AC_HOST && mem != AC_DEVICE) return set_error(AC_EINVAL, "ac_scan_batch: unknown memory kind");
    for (uint32_t i = 0; i < ni; ++i) memset(&outs[i], 0, sizeof(ac_result));
    const int device = as[0] ? as[0]->device : -1;
    for (uint32_t k = 0; k < na; ++k) {
        if (!as[k] || as[k]->device != device || device < 0)
            return set_error(AC_EINVAL, "ac_scan_batch: automata must be built on one device");
        if (as[k]->machine != AC_MACHINE_DFA)
            return set_error(AC_EINVAL, "ac_scan_batch: batches take failure-folded (DFA) machines");
    }
    for (uint32_t i = 0; i < ni; ++i) {
        const ac_batch_item &it = items[i];
        if (it.automaton >= na) return set_error(AC_EINVAL, "ac_scan_batch: item %u names automaton %u", i,
                                                 it.automaton);
        if (it.fmt != AC_U8 && it.fmt != AC_PACKED2) return set_error(AC_EINVAL, "ac_scan_batch: item %u format", i);
        if (it.fmt == AC_PACKED2 && as[it.automaton]->sigma != 4)
            return set_error(AC_EINVAL, "ac_scan_batch: item %u: packed text needs a 4-letter alphabet", i);
        if (it.n >= (1ull << 32)) return set_error(AC_ERANGE, "ac_scan_batch: item %u longer than 2^32-1", i);
        if (it.n && !it.text) return set_error(AC_EINVAL, "ac_scan_batch: item %u text is NULL", i);
    }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device && cudaSetDevice(device) != cudaSuccess)
        return set_error(AC_ECUDA, "ac_scan_batch: cannot use device %d", device);
    struct Restore {
        int d;
        ~Restore() {
            if (d >= 0) cudaSetDevice(d);
        }
    } restore{prev};
    cudaStream_t s = (cudaStream_t)stream;

    // alphabet classes: (format, symbol map) must be common within one launch
    std::vector<std::vector<uint32_t>> classes;
    std::vector<std::pair<int, const ac_automaton *>> class_rep;
    for (uint32_t i = 0; i < ni; ++i) {
        if (items[i].n == 0) {
            outs[i].num_patterns = as[items[i].automaton]->P;
            if (!(flags & AC_BATCH_NO_COUNTS)) {
                outs[i].counts = (uint64_t *)calloc(outs[i].num_patterns, 8);
                if (!outs[i].counts) return set_error(AC_ENOMEM, "ac_scan_batch: host counts");
            }
            continue;
        }
        const ac_automaton *a = as[items[i].automaton];
        size_t c = 0;
        for (; c < classes.size(); ++c) {
            const ac_automaton *r = class_rep[c].second;
            if (class_rep[c].first == items[i].fmt && r->sigma == a->sigma &&
                memcmp(r->sym_of_byte, a->sym_of_byte, 256) == 0)
                break;
        }
        if (c == classes.size()) {
            classes.emplace_back();
            class_rep.emplace_back(items[i].fmt, a);
        }
        classes[c].push_back(i);
    }

    int rc = AC_OK;
    for (size_t c = 0; c < classes.size() && rc == AC_OK; ++c) {
        const auto &idx = classes[c];
        const ac_automaton *rep = class_rep[c].second;
        const int fmt = class_rep[c].first;
        // byte texts of an alphabet with a free byte: one text per automaton
        const int sep = fmt == AC_U8 && !(flags & (AC_BATCH_GRAPH | AC_BATCH_ONE_LAUNCH)) ? separator_byte(rep) : -1;
        ac_log(2, "batch: %zu texts (%s), %s", idx.size(), fmt == AC_U8 ? "u8" : "packed",
               sep >= 0 ? "one text per automaton behind separator bytes" : "one-launch arena");
        if (sep >= 0) {
            rc = scan_segments(as, items, idx, mem, flags, (uint8_t)sep, s, outs);
            continue;
        }
        uint64_t total = 0;
        uint32_t warm = 0;
        for (uint32_t i : idx) {
            total += fmt == AC_U8 ? items[i].n : (items[i].n + 3) / 4;
            const uint32_t w = as[items[i].automaton]->max_len;
            warm = std::max(warm, fmt == AC_U8 ? w : (w + 3) / 4);
        }
        ac_scan_config cfg = rep->cfg;
        if (!cfg.threads) cfg.threads = 512;
        if (!cfg.chains) cfg.chains = 2;
        if (!cfg.stage_bytes) cfg.stage_bytes = (rep->K >= 8 || cfg.chains == 1) ? 32 : 16;
        auto init_plan = [&](Plan &P) {
            P.device = device;
            P.fmt = fmt;
            P.mem = mem;
            P.flags = flags;
            P.sigma = rep->sigma;
            P.acgt = rep->dna_acgt;
            memcpy(P.sym, rep->sym_of_byte, 256);
            P.placement = rep->placement;
            P.smem_cap = rep->smem_cap_bytes;
        };

        if (!(flags & AC_BATCH_GRAPH)) {
            Plan P;
            init_plan(P);
            P.pooled = true;
            P.pool_stream = s;
            const uint32_t L = rep->cfg.row_len ? (uint32_t)((rep->cfg.row_len / (fmt == AC_U8 ? 1 : 4) + 31) / 32 * 32)
                                                : default_row_bytes(total, warm, cfg, device);
            rc = layout(as, items, idx, std::max<uint32_t>(L, kStageBytes), cfg, flags, P);
            uint64_t cap = std::min<uint64_t>(total / 256 + 4096, 1ull << 26);
            for (int attempt = 0; attempt < 2 && rc == AC_OK; ++attempt) {
                rc = alloc_plan(P, cap);
                uint64_t M = 0;
                if (rc == AC_OK) rc = run_once(P, s, outs, &M);
                free_plan_buffers(P);
                if (rc != AC_OK || M <= cap) break;
                cap = M;
                if (attempt == 1) rc = set_error(AC_ERANGE, "ac_scan_batch: output beyond capacity after a retry");
            }
            continue;
        }

        // graph plan: keyed by automata, texts, lengths, formats, memory kind, flags
        PlanKey key;
        key.v.push_back((uintptr_t)mem);
        key.v.push_back((uintptr_t)flags);
        for (uint32_t i : idx) {
            key.v.push_back((uintptr_t)as[items[i].automaton]);
            key.v.push_back((uintptr_t)items[i].text);
            key.v.push_back((uintptr_t)items[i].n);
            key.v.push_back((uintptr_t)items[i].fmt);
        }
        std::lock_guard<std::mutex> lk(g_plan_mu);
        auto itp = g_plans.find(key);
        Plan *P = itp == g_plans.end() ? nullptr : itp->second.get();
        if (!P) {
            if (g_plans.size() >= kMaxPlans) {
                for (auto &kv : g_plans) free_plan_buffers(*kv.second);
                g_plans.clear();
            }
            auto up = std::make_unique<Plan>();
            P = up.get();
            init_plan(*P);
            // autotune row length x CTA shape on this batch
            const uint32_t L0 = default_row_bytes(total, warm, cfg, device);
            const ac_scan_config shapes[6] = {{0, 512, 2, 0, 32, 0}, {0, 512, 4, 0, 16, 0}, {0, 512, 2, 0, 16, 0},
                                              {0, 256, 4, 0, 32, 0}, {0, 512, 2, 0, 16, 48u << 10},
                                              {0, 512, 2, 0, 16, 16u << 10}};
            const uint32_t Ls[3] = {std::max<uint32_t>(kStageBytes, (L0 / 2 + 31) / 32 * 32), L0, L0 * 2};
            float best = 1e30f;
            ac_scan_config best_cfg = cfg;
            uint32_t best_L = L0;
            for (const auto &sh : shapes)
                for (uint32_t L : Ls) {
                    if (sh.smem_table_bytes && L != L0) continue;  // table size tried at the default row length
                    Plan T;
                    init_plan(T);
                    if (layout(as, items, idx, L, sh, flags | AC_BATCH_NO_COUNTS, T) != AC_OK) continue;
                    if (alloc_plan(T, 1 << 16) == AC_OK && copy_texts(T, s, false) == AC_OK) {
                        const float ms = time_scan(T, s);
                        if (ms < best) {
                            best = ms;
                            best_cfg = sh;
                            best_L = L;
                        }
                    }
                    cudaStreamSynchronize(s);
                    free_plan_buffers(T);
                }
            cudaGetLastError();
            rc = layout(as, items, idx, best_L, best_cfg, flags, *P);
            // size the output from one plain run
            uint64_t cap = std::min<uint64_t>(total / 256 + 4096, 1ull << 26);
            uint64_t M = 0;
            for (int attempt = 0; attempt < 2 && rc == AC_OK; ++attempt) {
                rc = alloc_plan(*P, cap);
                if (rc == AC_OK) rc = run_once(*P, s, outs, &M);
                if (rc != AC_OK || M <= cap) break;
                for (uint32_t i : idx) ac_result_free(&outs[i]);
                free_plan_buffers(*P);
                cap = M + M / 4 + 1024;
            }
            if (rc != AC_OK) {
                free_plan_buffers(*P);
                continue;
            }
            // pinned host buffers and the captured graph
            const uint32_t pni = (uint32_t)P->items.size();
            uint64_t stage_bytes = 0;
            for (uint64_t b : P->nbytes) stage_bytes += b;
            bool ok = cudaHostAlloc((void **)&P->h_rec, P->cap * 8, 0) == cudaSuccess &&
                      cudaHostAlloc((void **)&P->h_off, (pni + 1) * 8, 0) == cudaSuccess &&
                      cudaHostAlloc((void **)&P->h_num, 16, 0) == cudaSuccess &&
                      (!P->total_counts || cudaHostAlloc((void **)&P->h_counts, P->total_counts * 8, 0) == cudaSuccess) &&
                      (mem != AC_HOST || cudaHostAlloc((void **)&P->h_stage, stage_bytes, 0) == cudaSuccess);
            cudaGraph_t graph = nullptr;
            if (ok) {
                cudaStream_t cs;
                cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
                ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                int crc = ok ? copy_texts(*P, cs, mem == AC_HOST) : AC_ECUDA;
                if (crc == AC_OK) crc = device_sequence(*P, cs);
                if (crc == AC_OK) {
                    cudaMemcpyAsync(P->h_num, P->d_num, 16, cudaMemcpyDeviceToHost, cs);
                    cudaMemcpyAsync(P->h_rec, P->d_rec, P->cap * 8, cudaMemcpyDeviceToHost, cs);
                    cudaMemcpyAsync(P->h_off, P->d_off, (pni + 1) * 8, cudaMemcpyDeviceToHost, cs);
                    if (P->total_counts)
                        cudaMemcpyAsync(P->h_counts, P->d_counts, P->total_counts * 8, cudaMemcpyDeviceToHost, cs);
                }
                if (ok) ok = cudaStreamEndCapture(cs, &graph) == cudaSuccess && crc == AC_OK;
                if (ok) ok = cudaGraphInstantiate(&P->exec, graph, 0) == cudaSuccess;
                if (graph) cudaGraphDestroy(graph);
                cudaStreamDestroy(cs);
                cudaGetLastError();
            }
            if (!ok) P->exec = nullptr;  // the plan still works without a graph
            g_plans.emplace(key, std::move(up));
            continue;  // this call's results came from the plain run
        }
        // replay
        if (mem == AC_HOST && P->exec) {
            uint64_t off = 0;
            for (size_t i = 0; i < P->items.size(); ++i) {
                memcpy(P->h_stage + off, P->src[i], P->nbytes[i]);
                off += P->nbytes[i];
            }
        }
        if (P->exec) {
            if (cudaGraphLaunch(P->exec, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
                rc = set_error(AC_ECUDA, "ac_scan_batch: graph replay failed");
                continue;
            }
            if ((uint32_t)P->h_num[1]) {
                rc = set_error(AC_ETIMEDOUT, "ac_scan_batch: a device-side wait ran out");
                continue;
            }
            if (P->h_num[0] <= P->cap) {
                rc = split_results(*P, P->h_rec, P->h_off, P->total_counts ? P->h_counts : nullptr, outs);
                continue;
            }
        }
        // no graph, or more matches than the plan holds: plain run with a fitting capacity
        uint64_t M = 0;
        rc = run_once(*P, s, outs, &M);
        if (rc == AC_OK && M > P->cap) {
            for (uint32_t i : idx) ac_result_free(&outs[i]);
            Plan Q;
            init_plan(Q);
            Q.pooled = true;
            Q.pool_stream = s;
            rc = layout(as, items, idx, P->row_bytes, P->cfg, flags, Q);
            if (rc == AC_OK) rc = alloc_plan(Q, M);
            if (rc == AC_OK) rc = run_once(Q, s, outs, &M);
            cudaStreamSynchronize(s);
            free_plan_buffers(Q);
        }
    }
    if (rc != AC_OK)
        for (uint32_t i = 0; i < ni; ++i) ac_result_free(&outs[i]);
    return rc;
}

// Drop every kept batch plan (and its device memory).
extern "C" void ac_batch_release(void) {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    for (auto &kv : g_plans) free_plan_buffers(*kv.second);
    g_plans.clear();
}
