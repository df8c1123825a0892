// ac_tune: pick the scan configuration (CTA shape, shared-memory table size,
// symbols per lookup, row length) for an automaton by timing candidates on a
// real text, one coordinate at a time.
#include "ac_internal.h"

using namespace acgb;

extern "C" int ac_tune(ac_automaton *a, const uint8_t *d_text, uint64_t n, int fmt, void *stream,
                       ac_scan_config *chosen) {
    NvtxRange nvtx_range("ac_tune");
    if (!a || (!d_text && n)) return set_error(AC_EINVAL, "ac_tune: NULL argument");
    if (a->device < 0) return set_error(AC_EINVAL, "ac_tune: host-only automaton");
    if (fmt != AC_U8 && fmt != AC_PACKED2) return set_error(AC_EINVAL, "ac_tune: unknown format");
    if (fmt == AC_PACKED2 && a->sigma != 4) return set_error(AC_EINVAL, "ac_tune: packed text needs 4 letters");
    const uint64_t nbytes = fmt == AC_U8 ? n : (n + 3) / 4;
    if (nbytes < 64 || ((uintptr_t)d_text & 15))
        return set_error(AC_EINVAL, "ac_tune: the text must be 16-byte aligned and at least 64 bytes");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != a->device) cudaSetDevice(a->device);
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t cap = n / 256 + 4096;
    unsigned long long *num = (unsigned long long *)dev_alloc(16, s);
    unsigned long long *keys = (unsigned long long *)dev_alloc(cap * 8, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const ac_scan_config saved = a->cfg;
    int rc = (num && keys) ? AC_OK : set_error(AC_ENOMEM, "ac_tune: scratch");
    // time one configuration (best of 3); 1e30 if it cannot run
    auto timeit = [&](ac_scan_config c) -> float {
        ScanText t{d_text, n, fmt, nbytes};
        ScanOut o{keys, cap, num, nullptr, (uint32_t *)(num + 1)};
        float best_ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaMemsetAsync(num, 0, 16, s);
            cudaEventRecord(e0, s);
            if (launch_scan(a, t, o, c, s) != AC_OK) {
                cudaGetLastError();
                break;
            }
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = set_error(AC_ECUDA, "ac_tune: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            best_ms = std::min(best_ms, ms);
        }
        return best_ms;
    };
    // 1. kernel and CTA shape (threads x chains x stage bytes) at the default
    // row length and table
    ac_scan_config best{};
    float best_ms = 1e30f;
    auto try_shape = [&](uint32_t kernel, uint32_t t, uint32_t ch, uint32_t stage) {
        a->cfg = ac_scan_config{};
        a->cfg.threads = t;
        a->cfg.chains = ch;
        a->cfg.stage_bytes = stage;
        a->cfg.kernel = kernel;
        ac_scan_config c;
        default_config(a, n, fmt, &c);
        const float ms = timeit(c);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    };
    const uint32_t threads[2] = {256, 512}, chains[3] = {1, 2, 4}, stages[2] = {16, 32};
    for (int ti = 0; ti < 2 && rc == AC_OK; ++ti)
        for (int ci = 0; ci < 3 && rc == AC_OK; ++ci)
            for (int si = 0; si < 2 && rc == AC_OK; ++si) {
                if (stages[si] == 16 && chains[ci] == 1) continue;
                try_shape(AC_KERNEL_GENERAL, threads[ti], chains[ci], stages[si]);
            }
    // the lean kernel where it applies (its shapes; a candidate that does not apply times as 1e30)
    const uint32_t lean_shapes[4][2] = {{1024, 4}, {1024, 2}, {768, 4}, {512, 4}};
    for (int li = 0; li < 4 && rc == AC_OK; ++li)
        try_shape(AC_KERNEL_LEAN, lean_shapes[li][0], lean_shapes[li][1], 16);
    // the short-text kernel for texts up to 16 MiB (one thread per 16-byte row)
    if (nbytes <= (16ull << 20)) {
        const uint32_t short_threads[3] = {256, 512, 1024};
        for (int si = 0; si < 3 && rc == AC_OK; ++si) try_shape(AC_KERNEL_SHORT, short_threads[si], 1, 0);
    }
    // 2. shared-memory table size (the rest goes through L1/L2)
    const uint32_t caps[5] = {0, 96u << 10, 48u << 10, 16u << 10, 4u << 10};
    ac_scan_config base = best;
    for (int ki = 0; ki < 5 && rc == AC_OK; ++ki) {
        ac_scan_config c = base;
        c.smem_table_bytes = caps[ki];
        if (caps[ki] == base.smem_table_bytes) continue;
        const float ms = timeit(c);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    // 3. symbols per lookup (when the two-symbol table applies to this format)
    if (scan_stride(a, fmt, 2) == 2) {
        base = best;
        for (uint32_t stride = 1; stride <= 2 && rc == AC_OK; ++stride) {
            ac_scan_config c = base;
            c.stride = stride;
            if (stride == 2 && c.kernel != AC_KERNEL_GENERAL) {
                // two symbols per lookup run on the general kernel with its default shape
                a->cfg = ac_scan_config{};
                a->cfg.stride = 2;
                a->cfg.kernel = AC_KERNEL_GENERAL;
                default_config(a, n, fmt, &c);
            }
            const float ms = timeit(c);
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    }
    // 4. row length
    base = best;
    for (int li = 0; li < 2 && rc == AC_OK; ++li) {
        ac_scan_config c = base;
        c.row_len = li == 0 ? std::max<uint32_t>(64, base.row_len / 2) : base.row_len * 2;
        const float ms = timeit(c);
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaGetLastError();  // a candidate that did not fit (shared memory) is skipped
    a->cfg = (rc == AC_OK && best_ms < 1e29f) ? best : saved;
    if (chosen) *chosen = a->cfg;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(keys, s);
    dev_free(num, s);
    if (prev >= 0 && prev != a->device) cudaSetDevice(prev);
    return rc;
}
