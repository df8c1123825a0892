// ac_scan_noalloc: the asynchronous device-in, device-out scan for callers
// that must not allocate device memory.
//
// Who needs it: code that cannot call cudaMalloc / cudaMallocAsync at scan
// time — for example a process whose device memory was reserved up front by
// another allocator (a framework's caching allocator holding the whole
// budget), a latency-critical loop that cannot afford the implicit
// synchronisation or lock of an allocation, or an embedding application that
// forbids the library from touching the allocator at all. ac_scan_async
// takes its scratch from a stream-ordered pool; this variant takes it from
// one fixed array compiled into the library instead and allocates nothing.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes
// (about 8.1 MiB): the match counter and error word, the unsorted keys and
// the sort's second buffer for up to kNoAllocMaxMatches matches, the radix
// sort's temporary storage, and a small staging area for texts that are not
// 16-byte aligned or shorter than 64 bytes. A device holds this array from
// the first ac_scan_noalloc call on it (which loads this part of the
// library's device code and reserves the array) until the process exits, so
// make that first call at initialisation -- a call with n = 0 and cap = 0
// does it -- before the device's memory is committed elsewhere and before any
// stream capture.
#include <atomic>
#include <mutex>

#include "ac_internal.h"

namespace acgb {
namespace {

constexpr uint64_t kNoAllocMaxMatches = 1ull << 18;    // 262,144 match records per call
constexpr uint64_t kNoAllocTextBytes = 1ull << 16;     // staging for unaligned or short texts
constexpr uint64_t kNoAllocSortBytes = 4ull << 20;     // radix-sort temporary storage
constexpr uint64_t kHead = 256;                        // counter (8 B) + error word (4 B), padded
constexpr uint64_t kKeysOff = kHead;
constexpr uint64_t kAltOff = kKeysOff + kNoAllocMaxMatches * 8;
constexpr uint64_t kSortOff = kAltOff + kNoAllocMaxMatches * 8;
constexpr uint64_t kTextOff = kSortOff + kNoAllocSortBytes;
constexpr uint64_t kNoAllocScratchBytes = kTextOff + kNoAllocTextBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on each device, looked up with that
// device current (in host code the array's name is only a host-side handle).
// The library's code for a device is loaded lazily, so the first lookup on a
// device loads this file's module and reserves the array's memory then; it
// can fail (for instance with cudaErrorMemoryAllocation when another
// allocator already holds the device's memory). Only a successful lookup is
// kept: a failed one clears the runtime's error state, is reported, and the
// next call tries again.
constexpr int kMaxDevices = 64;
static std::mutex g_addr_mu;
static std::atomic<unsigned char *> g_addr[kMaxDevices];

unsigned char *scratch_on(int device, cudaError_t *err) {
    *err = cudaSuccess;
    if (unsigned char *p = g_addr[device].load(std::memory_order_acquire)) return p;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (unsigned char *p = g_addr[device].load(std::memory_order_acquire)) return p;
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();  // do not leave the error for another entry point's launch check
        *err = e != cudaSuccess ? e : cudaErrorInvalidSymbol;
        return nullptr;
    }
    g_addr[device].store((unsigned char *)p, std::memory_order_release);
    return (unsigned char *)p;
}

uint32_t value_bits(uint64_t x) {
    uint32_t b = 1;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

struct CurrentDevice {
    int prev = -1;
    bool ok = false;
    explicit CurrentDevice(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
            return;
        }
        ok = prev == d || cudaSetDevice(d) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    ~CurrentDevice() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace acgb

using namespace acgb;

extern "C" int ac_scan_noalloc(const ac_automaton *a, const uint8_t *d_text, uint64_t n, int fmt, void *stream,
                               ac_match *d_matches, uint64_t cap, uint64_t *d_num_matches, uint64_t *d_counts) {
    if (!a || !d_num_matches || (!d_text && n) || (!d_matches && cap))
        return set_error(AC_EINVAL, "ac_scan_noalloc: NULL argument");
    if (a->device < 0 || a->device >= kMaxDevices)
        return set_error(AC_EINVAL, "ac_scan_noalloc: automaton has no usable device");
    if (fmt != AC_U8 && fmt != AC_PACKED2) return set_error(AC_EINVAL, "ac_scan_noalloc: unknown format %d", fmt);
    if (fmt == AC_PACKED2 && a->sigma != 4)
        return set_error(AC_EINVAL, "ac_scan_noalloc: packed text needs a 4-letter alphabet");
    if (n >= (1ull << 32)) return set_error(AC_ERANGE, "ac_scan_noalloc: n is 2^32 or more");
    if (cap > kNoAllocMaxMatches)
        return set_error(AC_ERANGE, "ac_scan_noalloc: cap %llu is beyond the fixed scratch limit of %llu matches",
                         (unsigned long long)cap, (unsigned long long)kNoAllocMaxMatches);
    CurrentDevice dev(a->device);
    if (!dev.ok) return set_error(AC_ECUDA, "ac_scan_noalloc: cannot use device %d", a->device);
    cudaError_t e;
    unsigned char *base = scratch_on(a->device, &e);
    if (!base)
        return set_error(e == cudaErrorMemoryAllocation ? AC_ENOMEM : AC_ECUDA,
                         "ac_scan_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));

    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *num = (unsigned long long *)base;
    uint32_t *err = (uint32_t *)(base + 8);
    unsigned long long *keys = (unsigned long long *)(base + kKeysOff);
    unsigned long long *alt = (unsigned long long *)(base + kAltOff);
    void *sort_tmp = base + kSortOff;
    uint8_t *text_stage = base + kTextOff;

    // the counter and the error word must start at zero: the array keeps the
    // previous call's contents
    e = cudaMemsetAsync(base, 0, 16, s);
    if (e != cudaSuccess) return set_error(AC_ECUDA, "ac_scan_noalloc: %s", cudaGetErrorString(e));
    if (d_counts) {
        e = cudaMemsetAsync(d_counts, 0, (size_t)a->P * 8, s);
        if (e != cudaSuccess) return set_error(AC_ECUDA, "ac_scan_noalloc: %s", cudaGetErrorString(e));
    }
    const uint64_t nbytes = fmt == AC_U8 ? n : (n + 3) / 4;
    const uint64_t kcap = cap ? cap : 1;
    int rc = AC_OK;
    if (n) {
        const uint8_t *t = d_text;
        uint64_t readable = nbytes;
        if (((uintptr_t)d_text & 15) || nbytes < 64) {
            if (nbytes > kNoAllocTextBytes)
                return set_error(AC_EINVAL,
                                 "ac_scan_noalloc: a text over %llu bytes must be 16-byte aligned",
                                 (unsigned long long)kNoAllocTextBytes);
            if (nbytes < 64) {
                e = cudaMemsetAsync(text_stage, 0, 64, s);
                if (e != cudaSuccess) return set_error(AC_ECUDA, "ac_scan_noalloc: %s", cudaGetErrorString(e));
                readable = 64;
            }
            e = cudaMemcpyAsync(text_stage, d_text, nbytes, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return set_error(AC_ECUDA, "ac_scan_noalloc: %s", cudaGetErrorString(e));
            t = text_stage;
        }
        ac_scan_config cfg;
        default_config(a, n, fmt, &cfg);
        ScanText tx{t, n, fmt, readable};
        ScanOut o{keys, cap, num, (unsigned long long *)d_counts, err};
        rc = launch_scan(a, tx, o, cfg, s);
        if (rc) return rc;
    }
    unsigned long long *sorted = keys;
    if (cap) {
        rc = launch_pad_keys(keys, num, kcap, s);
        if (rc) return rc;
        const int end_bit = (int)std::min<uint32_t>(64, key_shift_for(a) + value_bits(n ? n - 1 : 0));
        size_t need = 0;
        rc = sort_keys(keys, alt, kcap, sort_begin_bit(a), end_bit, nullptr, &need, s, nullptr);
        if (rc) return rc;
        if (need > kNoAllocSortBytes)
            return set_error(AC_ERANGE, "ac_scan_noalloc: sort storage %zu bytes beyond the fixed limit", need);
        size_t have = kNoAllocSortBytes;
        rc = sort_keys(keys, alt, kcap, sort_begin_bit(a), end_bit, sort_tmp, &have, s, &sorted);
        if (rc) return rc;
    }
    return launch_keys_to_matches(sorted, num, cap, (uint32_t)key_shift_for(a), d_matches,
                                  (unsigned long long *)d_num_matches, err, s);
}
