// ac_probe_gather: the rate at which an SM array can make dependent random
// 4-byte table reads, for the rooflines of the scan kernels.
//
// Every symbol of an Aho-Corasick scan is one dependent lookup in the goto
// table (Section II.A; one lookup per symbol in the folded machine of
// Section III). Where that lookup lands decides the ceiling: shared memory
// (32 four-byte banks per SM, conflicts when lanes hit the same bank), L2
// (a random 32-byte sector per lookup) or HBM. This probe measures each on
// the device it runs on, with the same access pattern: every thread walks
// `chains` independent chains, each step reading the 4-byte word the
// previous one selects (x <- T[f(x)]), with no locality beyond what the
// table's size leaves. The table is filled with seeded pseudo-random words
// (splitmix64 of the index), so every step lands on a uniformly random word.
#include "ac_internal.h"

namespace acgb {
namespace {

__device__ __forceinline__ uint32_t mix64to32(uint64_t z) {
    // splitmix64 finaliser (Steele, Lea and Flood, 2014)
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (uint32_t)((z ^ (z >> 31)) >> 16);
}

__global__ void probe_fill_kernel(uint32_t *buf, uint64_t words, uint64_t seed) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x)
        buf[i] = mix64to32(i ^ (seed << 32));
}

__device__ __forceinline__ uint32_t ld_nc_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Global-memory table: `words` 4-byte entries; step: x = T[hi32(x * words)] + s.
template <int C>
__global__ void __launch_bounds__(1024, 1)
    probe_global_kernel(const uint32_t *__restrict__ buf, uint32_t words, uint32_t steps, uint32_t *sink) {
    uint32_t x[C];
#pragma unroll
    for (int j = 0; j < C; ++j) x[j] = mix64to32(((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * C + j);
    for (uint32_t s = 0; s < steps; ++s) {
#pragma unroll
        for (int j = 0; j < C; ++j) x[j] = ld_nc_u32(buf + __umulhi(x[j], words)) + s;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < C; ++j) acc ^= x[j];
    if (acc == 0x9e3779b9u) sink[0] = acc;  // keeps the chains live; practically never written
}

// Shared-memory table: the first `words` entries of the global table copied
// into shared memory; the same walk.
template <int C>
__global__ void __launch_bounds__(1024, 1)
    probe_shared_kernel(const uint32_t *__restrict__ buf, uint32_t words, uint32_t steps, uint32_t *sink) {
    extern __shared__ uint32_t tab[];
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) tab[i] = buf[i];
    __syncthreads();
    uint32_t x[C];
#pragma unroll
    for (int j = 0; j < C; ++j) x[j] = mix64to32(((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * C + j);
    for (uint32_t s = 0; s < steps; ++s) {
#pragma unroll
        for (int j = 0; j < C; ++j) x[j] = tab[__umulhi(x[j], words)] + s;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < C; ++j) acc ^= x[j];
    if (acc == 0x9e3779b9u) sink[0] = acc;
}

__global__ void probe_empty_kernel() {}

using ProbeFn = void (*)(const uint32_t *, uint32_t, uint32_t, uint32_t *);

ProbeFn pick(bool shared, uint32_t chains) {
    switch (chains) {
        case 1: return shared ? probe_shared_kernel<1> : probe_global_kernel<1>;
        case 2: return shared ? probe_shared_kernel<2> : probe_global_kernel<2>;
        case 4: return shared ? probe_shared_kernel<4> : probe_global_kernel<4>;
        case 8: return shared ? probe_shared_kernel<8> : probe_global_kernel<8>;
        default: return nullptr;
    }
}

}  // namespace
}  // namespace acgb

using namespace acgb;

extern "C" int ac_probe_gather(int device, uint64_t table_bytes, int shared, uint32_t threads, uint32_t chains,
                               uint32_t steps, ac_gather_probe *out) {
    if (!out) return set_error(AC_EINVAL, "ac_probe_gather: out is NULL");
    memset(out, 0, sizeof(*out));
    if (threads < 32 || threads > 1024 || threads % 32) return set_error(AC_EINVAL, "ac_probe_gather: threads");
    ProbeFn fn = pick(shared != 0, chains);
    if (!fn) return set_error(AC_EINVAL, "ac_probe_gather: chains per thread must be 1, 2, 4 or 8");
    const uint64_t words = table_bytes / 4;
    if (words < 32 || words >= (1ull << 32)) return set_error(AC_ERANGE, "ac_probe_gather: table size");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return set_error(AC_ECUDA, "ac_probe_gather: cannot use device %d", device);
    }
    int rc = AC_OK;
    uint32_t *buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    do {
        int sms = 0, smem_limit = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        cudaDeviceGetAttribute(&smem_limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
        const size_t smem = shared ? (size_t)words * 4 : 0;
        if (shared && smem > (size_t)smem_limit) {
            rc = set_error(AC_ERANGE, "ac_probe_gather: a %llu-byte table does not fit shared memory",
                           (unsigned long long)table_bytes);
            break;
        }
        if (cudaMalloc(&buf, words * 4 + 64) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(AC_ENOMEM, "ac_probe_gather: %llu bytes", (unsigned long long)table_bytes);
            break;
        }
        if (shared && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(AC_ECUDA, "ac_probe_gather: shared memory attribute");
            break;
        }
        probe_fill_kernel<<<sms * 4, 256>>>(buf, words, 0x5eedull);
        uint32_t *sink = buf + words;
        // warm-up: the table into L2 (when it fits) and the code loaded
        fn<<<sms, threads, smem>>>(buf, (uint32_t)words, std::max<uint32_t>(1, steps / 4), sink);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0);
        fn<<<sms, threads, smem>>>(buf, (uint32_t)words, steps, sink);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = set_error(AC_ECUDA, "ac_probe_gather: launch failed");
            break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        out->ms = ms;
        out->gathers = (double)sms * threads * chains * steps;
        out->gathers_per_s = ms > 0 ? out->gathers / (ms * 1e-3) : 0;
        out->chains_per_sm = threads * chains;
        out->sms = (uint32_t)sms;
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    cudaSetDevice(prev);
    return rc;
}

extern "C" int ac_probe_launch(void *stream, uint32_t launches, uint32_t blocks, uint32_t threads) {
    if (!launches || !blocks || !threads || threads > 1024)
        return set_error(AC_EINVAL, "ac_probe_launch: launches, blocks and threads must be positive, threads <= 1024");
    cudaStream_t s = (cudaStream_t)stream;
    for (uint32_t i = 0; i < launches; ++i) probe_empty_kernel<<<blocks, threads, 0, s>>>();
    if (cudaGetLastError() != cudaSuccess) return set_error(AC_ECUDA, "ac_probe_launch: launch failed");
    return AC_OK;
}
