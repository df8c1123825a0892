// Machine construction on the GPU (ac_build_opts.builder = AC_BUILDER_DEVICE):
// the same machine as the host build (build.cpp), state for state and entry
// for entry, for pattern sets large enough that building dominates (the
// paper's Section V measures build plus scan; Section III and reference [2]
// name building the machine as the cost that grows with the pattern set).
//
// Steps for one subset of patterns:
//  1. symbols: pattern bytes mapped to symbol codes;
//  2. sort: pattern indices sorted by their symbol strings (a shorter string
//     before its extensions, equal strings by pattern id) -- an LSD radix
//     sort over fixed-width keys of (symbol + 1) codes;
//  3. LCP of each pattern with its predecessor in that order. The goto
//     function's states are the distinct prefixes: pattern i (sorted order)
//     starts a new state at depth d exactly when lcp_i < d <= len_i. Counting
//     these starts depth by depth (row d of a depth x pattern matrix) with
//     one inclusive scan over the matrix numbers the states breadth-first,
//     and within a depth lexicographically -- the order in which a
//     breadth-first walk that visits children by symbol meets them, i.e. the
//     host build's numbering. The scan value at (d, i) is the id of the
//     depth-d state on pattern i's path;
//  4. goto edges, parent and symbol of every state, depth, own outputs;
//  5. failure function and fold of missing transitions (Section II.A's
//     failure transitions replaced by regular ones, the AC-opt machine of
//     Section III), one depth at a time: f(t) = next(f(parent), symbol),
//     next(s, c) = goto(s, c) if defined, else next(f(s), c); a state's
//     failure state is shallower, so its row is complete when needed;
//  6. output function, one depth at a time: |out(s)| = |own(s)| + |out(f(s))|,
//     offsets by a scan, then out(s) = merge of own(s) and out(f(s)), both
//     ascending; the output flag of every table entry.
// The tables are copied back into the host subset (the host view, the
// derived tables and the upload use them as for a host-built machine).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <chrono>
#include <cstring>

#include "ac_internal.h"

namespace acgb {
namespace {

constexpr uint32_t kNoState = 0xffffffffu;

// ------------------------------------------------------------------ kernels
__global__ void map_symbols_kernel(const uint8_t *__restrict__ bytes, uint64_t n, const uint8_t *__restrict__ sym_of,
                                   uint8_t *__restrict__ out) {
    __shared__ uint8_t map[256];
    for (uint32_t i = threadIdx.x; i < 256; i += blockDim.x) map[i] = sym_of[i];
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = map[bytes[i]];
}

// key word w of pattern i: symbols [w*per, (w+1)*per) as (code + 1) in `bits`
// bits each, most significant first; positions past the pattern's end are 0
__global__ void key_word_kernel(const uint8_t *__restrict__ syms, const uint64_t *__restrict__ off,
                                const uint32_t *__restrict__ len, const uint32_t *__restrict__ perm, uint32_t P,
                                uint32_t w, uint32_t per, uint32_t bits, unsigned long long *__restrict__ key) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const uint32_t j = perm[i];
    const uint8_t *s = syms + off[j];
    const uint32_t L = len[j];
    unsigned long long k = 0;
    for (uint32_t q = 0; q < per; ++q) {
        const uint32_t pos = w * per + q;
        const unsigned long long c = pos < L ? (unsigned long long)s[pos] + 1ull : 0ull;
        k = (k << bits) | c;
    }
    key[i] = k;
}

// lcp[i] = longest common prefix of sorted patterns i-1 and i (0 for i = 0);
// slen[i] = length of sorted pattern i
__global__ void lcp_kernel(const uint8_t *__restrict__ syms, const uint64_t *__restrict__ off,
                           const uint32_t *__restrict__ len, const uint32_t *__restrict__ perm, uint32_t P,
                           uint32_t *__restrict__ lcp, uint32_t *__restrict__ slen) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const uint32_t b = perm[i];
    slen[i] = len[b];
    if (i == 0) {
        lcp[0] = 0;
        return;
    }
    const uint32_t a = perm[i - 1];
    const uint8_t *x = syms + off[a], *y = syms + off[b];
    const uint32_t m = min(len[a], len[b]);
    uint32_t k = 0;
    while (k < m && x[k] == y[k]) ++k;
    lcp[i] = k;
}

// start[(d-1)*P + i] = 1 if sorted pattern i starts a new state at depth d
__global__ void starts_kernel(const uint32_t *__restrict__ lcp, const uint32_t *__restrict__ slen, uint32_t P,
                              uint32_t D, uint32_t *__restrict__ start) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= (uint64_t)P * D) return;
    const uint32_t d = (uint32_t)(t / P) + 1, i = (uint32_t)(t % P);
    start[t] = (lcp[i] < d && d <= slen[i]) ? 1u : 0u;
}

// goto edges, parent / symbol / depth of each state, own outputs: node(i, d) =
// inc[(d-1)*P + i] for d <= len_i (the root is 0)
__global__ void edges_kernel(const uint8_t *__restrict__ syms, const uint64_t *__restrict__ off,
                             const uint32_t *__restrict__ perm, const uint32_t *__restrict__ lcp,
                             const uint32_t *__restrict__ slen, const uint32_t *__restrict__ inc, uint32_t P,
                             uint32_t sigma, uint32_t *__restrict__ go, uint32_t *__restrict__ parent,
                             uint8_t *__restrict__ psym, uint32_t *__restrict__ depth, uint32_t *__restrict__ own_cnt,
                             uint32_t *__restrict__ own_first) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const uint32_t L = slen[i];
    const uint8_t *s = syms + off[perm[i]];
    // states from depth lcp_i + 1 on are new (started by this pattern)
    for (uint32_t d = lcp[i] + 1; d <= L; ++d) {
        const uint32_t node = inc[(uint64_t)(d - 1) * P + i];
        const uint32_t par = d == 1 ? 0u : inc[(uint64_t)(d - 2) * P + i];
        const uint32_t c = s[d - 1];
        go[(uint64_t)par * sigma + c] = node;
        parent[node] = par;
        psym[node] = (uint8_t)c;
        depth[node] = d;
    }
    // the pattern ends at node(i, L); equal patterns are adjacent in the order
    // and the first of them counts them all
    const uint32_t end = inc[(uint64_t)(L - 1) * P + i];
    if (i == 0 || lcp[i] < L || slen[i - 1] != L) {
        uint32_t k = 1;
        while (i + k < P && slen[i + k] == L && lcp[i + k] >= L) ++k;
        own_cnt[end] = k;
        own_first[end] = i;
    }
}

// depth-1 states and the root row
__global__ void root_kernel(const uint32_t *__restrict__ go, uint32_t sigma, uint32_t *__restrict__ table,
                            uint32_t *__restrict__ fail) {
    const uint32_t c = threadIdx.x;
    if (c >= sigma) return;
    const uint32_t t = go[c];
    table[c] = t == kNoState ? 0u : t;
    if (t != kNoState) fail[t] = 0;
    if (c == 0) fail[0] = 0;
}

// states [lo, hi) (one depth >= 1): failure state from the parent's failure
// state, then the folded row
__global__ void fold_kernel(uint32_t lo, uint32_t hi, uint32_t sigma, const uint32_t *__restrict__ go,
                            const uint32_t *__restrict__ parent, const uint8_t *__restrict__ psym,
                            uint32_t *__restrict__ table, uint32_t *__restrict__ fail) {
    const uint32_t s = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= hi) return;
    const uint32_t p = parent[s];
    const uint32_t f = p == 0 ? 0u : table[(uint64_t)fail[p] * sigma + psym[s]];
    fail[s] = f;
    const uint64_t rs = (uint64_t)s * sigma, rf = (uint64_t)f * sigma;
    for (uint32_t c = 0; c < sigma; ++c) {
        const uint32_t g = go[rs + c];
        table[rs + c] = g != kNoState ? g : table[rf + c];
    }
}

// |out(s)| = |own(s)| + |out(f(s))| for the states [lo, hi) of one depth
__global__ void out_count_kernel(uint32_t lo, uint32_t hi, const uint32_t *__restrict__ fail,
                                 const uint32_t *__restrict__ own_cnt, uint32_t *__restrict__ cnt) {
    const uint32_t s = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= hi) return;
    cnt[s] = own_cnt[s] + (s == 0 ? 0u : cnt[fail[s]]);
}

// out(s) = merge(own(s), out(f(s))), both ascending, for the states [lo, hi)
__global__ void out_fill_kernel(uint32_t lo, uint32_t hi, const uint32_t *__restrict__ fail,
                                const uint32_t *__restrict__ own_cnt, const uint32_t *__restrict__ own_first,
                                const uint32_t *__restrict__ perm, const uint32_t *__restrict__ out_off,
                                uint32_t *__restrict__ out_ids, uint32_t id_lo) {
    const uint32_t s = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= hi) return;
    const uint32_t oe = own_cnt[s];
    const uint32_t *own = perm + (oe ? own_first[s] : 0u);
    const uint32_t f = fail[s];
    const uint32_t fb = out_off[f], fe = s == 0 ? fb : out_off[f + 1];
    uint32_t a = 0, b = fb, w = out_off[s];
    while (a < oe && b < fe) {
        const uint32_t x = own[a] + id_lo, y = out_ids[b];
        if (x <= y) {
            out_ids[w++] = x;
            ++a;
        } else {
            out_ids[w++] = y;
            ++b;
        }
    }
    while (a < oe) out_ids[w++] = own[a++] + id_lo;
    while (b < fe) out_ids[w++] = out_ids[b++];
}

// entry flag: the next state's output is not empty
__global__ void flag_kernel(uint64_t n, const uint32_t *__restrict__ cnt, uint32_t *__restrict__ table) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t t = table[i];
        table[i] = t | (cnt[t] ? kFlag : 0u);
    }
}

__global__ void iota_kernel(uint32_t *p, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

template <typename T>
__global__ void gather_kernel(const T *__restrict__ src, const uint32_t *__restrict__ idx, uint32_t n,
                              T *__restrict__ dst) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

unsigned blocks_for(uint64_t n, unsigned t = 256) { return (unsigned)std::max<uint64_t>(1, (n + t - 1) / t); }

// RAII device buffers of one build
struct DevBufs {
    std::vector<void *> ptrs;
    template <typename T>
    T *get(size_t count) {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    ~DevBufs() {
        for (void *p : ptrs) cudaFree(p);
    }
};

}  // namespace

#define GB_CK(call, what)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            why = std::string(what) + ": " + cudaGetErrorString(e_);                            \
            return AC_ECUDA;                                                                    \
        }                                                                                       \
    } while (0)
#define GB_ALLOC(ptr, T, n)                                                                     \
    do {                                                                                        \
        ptr = bufs.get<T>(n);                                                                   \
        if (!ptr) {                                                                             \
            why = "device allocation failed";                                                   \
            return AC_ENOMEM;                                                                   \
        }                                                                                       \
    } while (0)

// Build subset [lo, hi) of the patterns on device `device` (current) into S,
// exactly as build_subset does on the host.
int build_subset_device(const uint8_t *const *pats, const uint32_t *lens, uint32_t lo, uint32_t hi,
                        const uint8_t *sym_of_byte, uint32_t sigma, HostSubset &S, std::string &why) {
    S.id_lo = lo;
    S.id_hi = hi;
    const uint32_t P = hi - lo;
    uint64_t chars = 0;
    uint32_t D = 0;
    for (uint32_t j = lo; j < hi; ++j) {
        chars += lens[j];
        D = std::max(D, lens[j]);
    }
    S.max_len = D;
    cudaStream_t st = 0;
    DevBufs bufs;

    // 1. pattern bytes (concatenated on the host, the input's layout) -> symbols
    std::vector<uint8_t> h_bytes(chars);
    std::vector<uint64_t> h_off(P);
    std::vector<uint32_t> h_len(P);
    {
        uint64_t o = 0;
        for (uint32_t j = 0; j < P; ++j) {
            h_off[j] = o;
            h_len[j] = lens[lo + j];
            memcpy(h_bytes.data() + o, pats[lo + j], lens[lo + j]);
            o += lens[lo + j];
        }
    }
    uint8_t *d_bytes, *d_syms, *d_map;
    uint64_t *d_off;
    uint32_t *d_len;
    GB_ALLOC(d_bytes, uint8_t, chars);
    GB_ALLOC(d_syms, uint8_t, chars);
    GB_ALLOC(d_map, uint8_t, 256);
    GB_ALLOC(d_off, uint64_t, P);
    GB_ALLOC(d_len, uint32_t, P);
    GB_CK(cudaMemcpyAsync(d_bytes, h_bytes.data(), chars, cudaMemcpyHostToDevice, st), "build: copy patterns");
    GB_CK(cudaMemcpyAsync(d_off, h_off.data(), P * 8ull, cudaMemcpyHostToDevice, st), "build: copy offsets");
    GB_CK(cudaMemcpyAsync(d_len, h_len.data(), P * 4ull, cudaMemcpyHostToDevice, st), "build: copy lengths");
    GB_CK(cudaMemcpyAsync(d_map, sym_of_byte, 256, cudaMemcpyHostToDevice, st), "build: copy symbol map");
    map_symbols_kernel<<<blocks_for(chars), 256, 0, st>>>(d_bytes, chars, d_map, d_syms);

    // 2. sort pattern indices by symbol string (LSD over key words; stable)
    uint32_t bits = 1;
    while ((1u << bits) < sigma + 1) ++bits;
    const uint32_t per = 64 / bits, W = (D + per - 1) / per;
    uint32_t *perm, *perm2;
    unsigned long long *key, *key2;
    GB_ALLOC(perm, uint32_t, P);
    GB_ALLOC(perm2, uint32_t, P);
    GB_ALLOC(key, unsigned long long, P);
    GB_ALLOC(key2, unsigned long long, P);
    iota_kernel<<<blocks_for(P), 256, 0, st>>>(perm, P);
    size_t temp_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, key, key2, perm, perm2, (int)P, 0, 64, st);
    void *temp;
    GB_ALLOC(temp, uint8_t, temp_bytes);
    for (uint32_t w = W; w-- > 0;) {
        key_word_kernel<<<blocks_for(P), 256, 0, st>>>(d_syms, d_off, d_len, perm, P, w, per, bits, key);
        GB_CK(cub::DeviceRadixSort::SortPairs(temp, temp_bytes, key, key2, perm, perm2, (int)P, 0, (int)(per * bits),
                                              st),
              "build: sort");
        std::swap(perm, perm2);
    }

    // 3. LCP with the predecessor, node starts per depth, one scan
    uint32_t *lcp, *slen, *start, *inc;
    const uint64_t DP = (uint64_t)D * P;
    GB_ALLOC(lcp, uint32_t, P);
    GB_ALLOC(slen, uint32_t, P);
    GB_ALLOC(start, uint32_t, DP);
    GB_ALLOC(inc, uint32_t, DP);
    lcp_kernel<<<blocks_for(P), 256, 0, st>>>(d_syms, d_off, d_len, perm, P, lcp, slen);
    starts_kernel<<<blocks_for(DP), 256, 0, st>>>(lcp, slen, P, D, start);
    if (DP >= (1ull << 31)) {
        why = "pattern set too large for the device build (depth x patterns >= 2^31)";
        return AC_ERANGE;
    }
    size_t scan_bytes = 0;
    cub::DeviceScan::InclusiveSum(nullptr, scan_bytes, start, inc, (int)DP, st);
    void *scan_temp;
    GB_ALLOC(scan_temp, uint8_t, scan_bytes);
    GB_CK(cub::DeviceScan::InclusiveSum(scan_temp, scan_bytes, start, inc, (int)DP, st), "build: scan");
    // states = 1 + total starts; level sizes from the row ends of the scan
    std::vector<uint32_t> row_end(D);
    for (uint32_t d = 0; d < D; ++d)
        GB_CK(cudaMemcpyAsync(&row_end[d], inc + (uint64_t)d * P + (P - 1), 4, cudaMemcpyDeviceToHost, st),
              "build: level sizes");
    GB_CK(cudaStreamSynchronize(st), "build: trie");
    const uint64_t N64 = 1ull + (D ? row_end[D - 1] : 0u);
    if (N64 >= (uint64_t)kStateMask) {
        why = "more than 2^31-1 states in one subset";
        return AC_ERANGE;
    }
    const uint32_t N = (uint32_t)N64;
    // states of depth d: [level[d], level[d+1])
    std::vector<uint32_t> level(D + 2);
    level[0] = 0;
    level[1] = 1;
    for (uint32_t d = 1; d <= D; ++d) level[d + 1] = 1 + row_end[d - 1];

    // 4. goto edges, parents, own outputs
    uint32_t *go, *parent, *depth, *own_cnt, *own_first, *table, *fail, *cnt, *out_off;
    uint8_t *psym;
    GB_ALLOC(go, uint32_t, (uint64_t)N * sigma);
    GB_ALLOC(parent, uint32_t, N);
    GB_ALLOC(psym, uint8_t, N);
    GB_ALLOC(depth, uint32_t, N);
    GB_ALLOC(own_cnt, uint32_t, N);
    GB_ALLOC(own_first, uint32_t, N);
    GB_ALLOC(table, uint32_t, (uint64_t)N * sigma);
    GB_ALLOC(fail, uint32_t, N);
    GB_ALLOC(cnt, uint32_t, N);
    GB_ALLOC(out_off, uint32_t, N + 1);
    GB_CK(cudaMemsetAsync(go, 0xff, (uint64_t)N * sigma * 4, st), "build: memset");
    GB_CK(cudaMemsetAsync(own_cnt, 0, N * 4ull, st), "build: memset");
    GB_CK(cudaMemsetAsync(depth, 0, N * 4ull, st), "build: memset");
    GB_CK(cudaMemsetAsync(parent, 0, N * 4ull, st), "build: memset");
    edges_kernel<<<blocks_for(P), 256, 0, st>>>(d_syms, d_off, perm, lcp, slen, inc, P, sigma, go, parent, psym,
                                                 depth, own_cnt, own_first);

    // 5. failure function and fold, one depth at a time
    root_kernel<<<1, 256, 0, st>>>(go, sigma, table, fail);
    for (uint32_t d = 1; d <= D; ++d) {
        const uint32_t a = level[d], b = level[d + 1];
        if (b > a) fold_kernel<<<blocks_for(b - a), 256, 0, st>>>(a, b, sigma, go, parent, psym, table, fail);
    }

    // 6. output function
    for (uint32_t d = 0; d <= D; ++d) {
        const uint32_t a = level[d], b = level[d + 1];
        if (b > a) out_count_kernel<<<blocks_for(b - a), 256, 0, st>>>(a, b, fail, own_cnt, cnt);
    }
    GB_CK(cudaMemsetAsync(out_off, 0, 4, st), "build: memset");
    size_t scan2 = 0;
    cub::DeviceScan::InclusiveSum(nullptr, scan2, cnt, out_off + 1, (int)N, st);
    void *scan2_temp;
    GB_ALLOC(scan2_temp, uint8_t, scan2);
    GB_CK(cub::DeviceScan::InclusiveSum(scan2_temp, scan2, cnt, out_off + 1, (int)N, st), "build: output scan");
    uint32_t M = 0;
    GB_CK(cudaMemcpyAsync(&M, out_off + N, 4, cudaMemcpyDeviceToHost, st), "build: output size");
    GB_CK(cudaStreamSynchronize(st), "build: outputs");
    uint32_t *out_ids;
    GB_ALLOC(out_ids, uint32_t, M);
    for (uint32_t d = 0; d <= D; ++d) {
        const uint32_t a = level[d], b = level[d + 1];
        if (b > a)
            out_fill_kernel<<<blocks_for(b - a), 256, 0, st>>>(a, b, fail, own_cnt, own_first, perm, out_off,
                                                                out_ids, lo);
    }
    flag_kernel<<<blocks_for((uint64_t)N * sigma), 256, 0, st>>>((uint64_t)N * sigma, cnt, table);
    GB_CK(cudaGetLastError(), "build: launch");

    // copy back
    S.states = N;
    S.table.resize((size_t)N * sigma);
    S.fail.resize(N);
    S.depth.resize(N);
    S.out_off.resize((size_t)N + 1);
    S.out_ids.resize(M);
    GB_CK(cudaMemcpyAsync(S.table.data(), table, (uint64_t)N * sigma * 4, cudaMemcpyDeviceToHost, st), "build: copy");
    GB_CK(cudaMemcpyAsync(S.fail.data(), fail, N * 4ull, cudaMemcpyDeviceToHost, st), "build: copy");
    GB_CK(cudaMemcpyAsync(S.depth.data(), depth, N * 4ull, cudaMemcpyDeviceToHost, st), "build: copy");
    GB_CK(cudaMemcpyAsync(S.out_off.data(), out_off, (N + 1ull) * 4, cudaMemcpyDeviceToHost, st), "build: copy");
    if (M) GB_CK(cudaMemcpyAsync(S.out_ids.data(), out_ids, M * 4ull, cudaMemcpyDeviceToHost, st), "build: copy");
    GB_CK(cudaStreamSynchronize(st), "build: copy back");
    return AC_OK;
}

}  // namespace acgb
