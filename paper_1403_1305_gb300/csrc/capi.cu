// C ABI entry points of libacgb300 (declared in include/ac.h): automaton
// lifecycle, synchronous and asynchronous scans, results, errors.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <chrono>
#include <mutex>

#include "ac_internal.h"

namespace acgb {

// ------------------------------------------------------------------ errors
static thread_local char g_last_error[512] = "";

// AC_LOG (environment, read once): 0 or unset = silent, 1 = every error
// message on stderr, 2 = also one line per build, scan plan and batch path.
int log_level() {
    static std::once_flag once;
    static int level = 0;
    std::call_once(once, [] {
        const char *v = getenv("AC_LOG");
        level = v ? atoi(v) : 0;
    });
    return level;
}

void ac_log(int level, const char *fmt, ...) {
    if (log_level() < level) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    fprintf(stderr, "acgb300: %s\n", buf);
}

int set_error(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    if (log_level() >= 1) fprintf(stderr, "acgb300: error %d: %s\n", code, g_last_error);
    return code;
}

static int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(AC_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(AC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

static void log_plan(const ac_automaton *a, uint64_t n, int fmt, const ac_scan_config &c) {
    if (log_level() < 2) return;
    static const char *kName[4] = {"auto", "general", "lean", "short"};
    ac_log(2, "scan: %llu symbols (%s) on %u subsets: %s kernel, rows of %u symbols, %u threads x %u chains",
           (unsigned long long)n, fmt == AC_U8 ? "u8" : "packed", a->K, kName[c.kernel & 3], c.row_len, c.threads,
           c.chains);
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ------------------------------------------------------------------ device memory
// Scratch comes from one stream-ordered pool per device that keeps freed
// memory reserved (release threshold = max), so steady-state scans allocate
// without a device synchronisation.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

static cudaMemPool_t pool_for(int device) {
    if (device < 0 || device >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[device]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        g_pools[device] = p;
    }
    return g_pools[device];
}

// Fault injection for tests (environment, read once): AC_FAULT_ALLOC=N lets
// N device scratch allocations succeed and fails every later one, so the
// calls' out-of-memory paths (AC_ENOMEM, nothing launched on a missing
// buffer) run without a real shortage.
static bool scratch_allowed() {
    static std::once_flag once;
    static bool injected = false;
    static std::atomic<int64_t> left{0};
    std::call_once(once, [] {
        const char *v = getenv("AC_FAULT_ALLOC");
        if (v && *v) {
            injected = true;
            left = std::max<int64_t>(0, atoll(v));
        }
    });
    return !injected || left.fetch_sub(1) > 0;
}

// Limit of the bounded device-side waits (mbarrier waits on TMA copies) of a
// scan launch: 2 s. Fault injection for tests (environment, read once):
// AC_FAULT_WAIT=N gives the next N launches with such waits a limit of 0, so
// each gives up at its first wait, sets the error word, lets the copies it
// issued land and exits (the call reports AC_ETIMEDOUT); later launches get
// the normal limit. No wait is left unbounded and nothing faults.
uint64_t wait_limit_ns() {
    static std::once_flag once;
    static std::atomic<int64_t> left{0};
    std::call_once(once, [] {
        const char *v = getenv("AC_FAULT_WAIT");
        if (v && *v) left = std::max<int64_t>(0, atoll(v));
    });
    if (left.load(std::memory_order_relaxed) > 0 && left.fetch_sub(1) > 0) return 0;
    return 2000000000ull;
}

void *dev_alloc(size_t bytes, cudaStream_t stream) {
    if (!scratch_allowed()) return nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPool_t p = pool_for(dev);
    void *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = p ? cudaMallocFromPoolAsync(&ptr, bytes, p, stream) : cudaMallocAsync(&ptr, bytes, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return ptr;
}

void dev_free(void *p, cudaStream_t stream) {
    if (p) cudaFreeAsync(p, stream);
}

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            prev = -1;
            ok = false;
            cudaGetLastError();
            return;
        }
        if (prev != d && cudaSetDevice(d) != cudaSuccess) {
            ok = false;
            cudaGetLastError();
        }
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Scratch allocations released (stream-ordered) when the scope ends.
struct Scratch {
    cudaStream_t s;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t st) : s(st) {}
    void *get(size_t bytes) {
        void *p = dev_alloc(bytes, s);
        if (p) ptrs.push_back(p);
        return p;
    }
    void release(void *p) {
        for (auto &q : ptrs)
            if (q == p) {
                dev_free(q, s);
                q = nullptr;
            }
    }
    ~Scratch() {
        for (void *p : ptrs) dev_free(p, s);
    }
};

static void free_device(ac_automaton *a) {
    if (a->device < 0) return;
    DeviceGuard g(a->device);
    for (auto &d : a->dsubs) {
        cudaFree(d.table);
        cudaFree(d.table2);
        cudaFree(d.table16);
        cudaFree(d.table_e16);
        cudaFree(d.out_off);
        cudaFree(d.out_ids);
    }
    a->dsubs.clear();
    if (a->d_desc) cudaFree(a->d_desc);
    a->d_desc = nullptr;
}

static int upload(ac_automaton *a) {
    auto t0 = std::chrono::steady_clock::now();
    DeviceGuard g(a->device);
    if (!g.ok) return set_error(AC_ECUDA, "ac_build: cannot use device %d", a->device);
    a->dsubs.assign(a->K, DeviceSubset());
    a->h_desc.assign(a->K, SubsetDev());
    for (uint32_t k = 0; k < a->K; ++k) {
        const HostSubset &h = a->subs[k];
        DeviceSubset &d = a->dsubs[k];
        size_t tb = h.table.size() * 4, ob = h.out_off.size() * 4, ib = std::max<size_t>(4, h.out_ids.size() * 4);
        CK(cudaMalloc(&d.table, tb), "ac_build: table");
        CK(cudaMalloc(&d.out_off, ob), "ac_build: output offsets");
        CK(cudaMalloc(&d.out_ids, ib), "ac_build: output ids");
        CK(cudaMemcpy(d.table, h.table.data(), tb, cudaMemcpyHostToDevice), "ac_build: copy");
        CK(cudaMemcpy(d.out_off, h.out_off.data(), ob, cudaMemcpyHostToDevice), "ac_build: copy");
        if (!h.out_ids.empty())
            CK(cudaMemcpy(d.out_ids, h.out_ids.data(), h.out_ids.size() * 4, cudaMemcpyHostToDevice),
               "ac_build: copy");
        if (!h.table2.empty()) {
            CK(cudaMalloc(&d.table2, h.table2.size() * 4), "ac_build: two-symbol table");
            CK(cudaMemcpy(d.table2, h.table2.data(), h.table2.size() * 4, cudaMemcpyHostToDevice), "ac_build: copy");
        }
        if (!h.table16.empty()) {
            CK(cudaMalloc(&d.table16, h.table16.size() * 2), "ac_build: 16-bit prefix");
            CK(cudaMemcpy(d.table16, h.table16.data(), h.table16.size() * 2, cudaMemcpyHostToDevice), "ac_build: copy");
        }
        if (!h.table_e16.empty()) {
            CK(cudaMalloc(&d.table_e16, h.table_e16.size() * 2), "ac_build: escape-coded 16-bit prefix");
            CK(cudaMemcpy(d.table_e16, h.table_e16.data(), h.table_e16.size() * 2, cudaMemcpyHostToDevice),
               "ac_build: copy");
        }
        SubsetDev &s = a->h_desc[k];
        s.table = d.table;
        s.table_e16 = d.table_e16;
        s.rows_e16 = d.table_e16 ? h.rows_e16 : 0;
        s.table2 = d.table2;
        s.table16 = d.table16;
        s.rows16 = d.table16 ? h.rows16 : 0;
        s.out_off = d.out_off;
        s.out_ids = d.out_ids;
        s.states = h.states;
        s.smem_states = 0;
        s.warm = h.max_len ? h.max_len - 1 : 0;
        s.id_lo = h.id_lo;
    }
    CK(cudaMalloc(&a->d_desc, sizeof(SubsetDev) * a->K), "ac_build: descriptors");
    CK(cudaMemcpy(a->d_desc, a->h_desc.data(), sizeof(SubsetDev) * a->K, cudaMemcpyHostToDevice),
       "ac_build: descriptors");
    // the scratch pool and the launches' one-time state exist before the first
    // scan, which may be under stream capture (where creating them is refused)
    (void)pool_for(a->device);
    prime_scan_state();
    a->upload_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return AC_OK;
}

// Placement SMEM: every table must fit the general kernel's shared-memory
// room (the lean kernel steps aside when its own is smaller).
static int check_smem_placement(ac_automaton *a) {
    if (a->placement != AC_PLACE_SMEM) return AC_OK;
    ac_scan_config c{};
    const ac_scan_config user = a->cfg;
    a->cfg.kernel = AC_KERNEL_GENERAL;
    default_config(a, 1, AC_U8, &c);
    a->cfg = user;
    int limit = scan_smem_limit(a->device);
    uint64_t avail = (uint64_t)std::max(0, limit - (int)scan_stage_bytes_per_cta(c) - 64);
    if (a->smem_cap_bytes && a->smem_cap_bytes < avail) avail = a->smem_cap_bytes;
    for (auto &s : a->subs)
        if ((uint64_t)s.states * 4 * a->sigma > avail)
            return set_error(AC_ERANGE, "placement SMEM, but a table of %u states does not fit", s.states);
    return AC_OK;
}

static uint32_t bits_for(uint64_t x) {
    uint32_t b = 1;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

static int check_scan_args(const ac_automaton *a, uint64_t n, int fmt) {
    if (!a) return set_error(AC_EINVAL, "scan: automaton is NULL");
    if (a->device < 0) return set_error(AC_EINVAL, "scan: automaton was built for the host only");
    if (fmt != AC_U8 && fmt != AC_PACKED2) return set_error(AC_EINVAL, "scan: unknown text format %d", fmt);
    if (fmt == AC_PACKED2 && a->sigma != 4)
        return set_error(AC_EINVAL, "scan: 2-bit packed text needs a 4-letter alphabet (have %u)", a->sigma);
    if (n >= (1ull << 32)) return set_error(AC_ERANGE, "scan: n = %llu symbols, the limit is 2^32-1",
                                            (unsigned long long)n);
    return AC_OK;
}

static uint64_t text_bytes(uint64_t n, int fmt) { return fmt == AC_U8 ? n : (n + 3) / 4; }

// Entries of the lean kernel's queue of stages with matches (split evenly
// between the launch's warps): one per 256 symbols and at least 65,536, at
// most one per 16-byte stage; stages beyond a warp's part are walked again
// in place, which is exact too.
uint64_t emit_queue_cap(uint64_t n, int fmt) {
    return std::min<uint64_t>(text_bytes(n, fmt) / 16 + 1, n / 256 + 65536);
}

// Device copy of the text at a 16-byte aligned address. Texts shorter than
// 64 bytes are copied into a zero-padded 64-byte buffer (the scan reads whole
// 32-byte stages of full rows); *readable receives the bytes that may be read.
static int stage_text(const uint8_t *text, uint64_t nbytes, int mem, cudaStream_t s, Scratch &sc,
                      const uint8_t **d_text, uint64_t *readable) {
    *readable = nbytes;
    if (mem == AC_DEVICE && ((uintptr_t)text & 15) == 0 && nbytes >= 64) {
        *d_text = text;
        return AC_OK;
    }
    const uint64_t alloc = std::max<uint64_t>(64, (nbytes + 15) & ~15ull);
    uint8_t *buf = (uint8_t *)sc.get(alloc);
    if (!buf) return set_error(AC_ENOMEM, "scan: device text buffer of %llu bytes", (unsigned long long)nbytes);
    if (nbytes < 64) CK(cudaMemsetAsync(buf, 0, 64, s), "scan: text padding");
    CK(cudaMemcpyAsync(buf, text, nbytes, mem == AC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s),
       "scan: text copy");
    *d_text = buf;
    if (nbytes < 64) *readable = 64;
    return AC_OK;
}

// Host texts of at least this many bytes are copied in pieces that overlap the scan.
constexpr uint64_t kPipeMinBytes = 32ull << 20;

// The library's copy stream of the current device (one per device, created on
// first use; never destroyed).
static cudaStream_t copy_stream() {
    static std::mutex mu;
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
        streams[dev] = nullptr;
    return streams[dev];
}

// Copy host text[0, t.n) into d_text piece by piece on the copy stream and
// scan each piece's rows on stream s as soon as the piece has landed: the
// rows of one launch read the bytes before them (their warm-up) from pieces
// copied earlier, and every launch uses the same row geometry, so the union
// of the launches is exactly one scan of the text.
static int pipelined_scan(const ac_automaton *a, const uint8_t *host, const uint8_t *d_text, const ScanText &t,
                          const ScanOut &o, const ac_scan_config &cfg, cudaStream_t s) {
    const uint64_t nbytes = text_bytes(t.n, t.fmt);
    const uint64_t rb = scan_row_bytes(cfg, t.fmt, t.readable);
    const uint64_t full_rows = t.readable / rb;
    const uint64_t num_rows = full_rows + (nbytes > full_rows * rb ? 1 : 0);
    // a piece's scan takes at least one row block's latency (~0.1 ms); 8
    // pieces of at least 32 MiB keep each scan within the next piece's copy
    const uint64_t piece_bytes = std::max<uint64_t>(32ull << 20, (nbytes + 7) / 8);
    const uint64_t piece_rows = std::max<uint64_t>(1, piece_bytes / rb);
    cudaStream_t cs = copy_stream();
    if (!cs) return set_error(AC_ECUDA, "ac_scan: no copy stream");
    std::vector<cudaEvent_t> evs;
    auto done = [&](int rc) {
        // s waits for everything this call put on the copy stream (the text
        // buffer is released in the order of s), also after an error
        cudaEvent_t last;
        if (cudaEventCreateWithFlags(&last, cudaEventDisableTiming) == cudaSuccess) {
            cudaEventRecord(last, cs);
            cudaStreamWaitEvent(s, last, 0);
            cudaEventDestroy(last);
        }
        for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
        return rc;
    };
    // the copy stream starts after the text buffer's allocation on s
    cudaEvent_t start;
    if (cudaEventCreateWithFlags(&start, cudaEventDisableTiming) != cudaSuccess)
        return set_error(AC_ECUDA, "ac_scan: event");
    evs.push_back(start);
    if (cudaEventRecord(start, s) != cudaSuccess || cudaStreamWaitEvent(cs, start, 0) != cudaSuccess)
        return done(set_error(AC_ECUDA, "ac_scan: copy stream order"));
    for (uint64_t r0 = 0; r0 < num_rows; r0 += piece_rows) {
        const uint64_t r1 = std::min(num_rows, r0 + piece_rows);
        const uint64_t b0 = r0 * rb, b1 = r1 == num_rows ? nbytes : std::min(nbytes, r1 * rb);
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return done(set_error(AC_ECUDA, "ac_scan: event"));
        evs.push_back(ev);
        if (b1 > b0 &&
            cudaMemcpyAsync((void *)(d_text + b0), host + b0, b1 - b0, cudaMemcpyHostToDevice, cs) != cudaSuccess)
            return done(set_error(AC_ECUDA, "ac_scan: text copy"));
        if (cudaEventRecord(ev, cs) != cudaSuccess || cudaStreamWaitEvent(s, ev, 0) != cudaSuccess)
            return done(set_error(AC_ECUDA, "ac_scan: piece order"));
        ScanText piece = t;
        piece.row_begin = r0;
        piece.row_end = r1;
        const int rc = launch_scan(a, piece, o, cfg, s);
        if (rc) return done(rc);
    }
    return done(AC_OK);
}

}  // namespace acgb

using namespace acgb;

// ====================================================================== C ABI
extern "C" {

int ac_version(void) { return 10000; }

const char *ac_strerror(int code) {
    switch (code) {
        case AC_OK: return "ok";
        case AC_EINVAL: return "invalid argument";
        case AC_ENOMEM: return "out of memory";
        case AC_ERANGE: return "size out of range";
        case AC_ECUDA: return "CUDA error";
        case AC_ETIMEDOUT: return "timed out";
        case AC_EAGAIN: return "not ready";
        case AC_EBUSY: return "busy";
        default: return "unknown error";
    }
}

const char *ac_last_error(void) { return g_last_error; }

int ac_build(const uint8_t *const *pats, const uint32_t *lens, uint32_t P, const ac_build_opts *opts,
             ac_automaton **out) {
    NvtxRange nvtx_range("ac_build");
    if (!out) return set_error(AC_EINVAL, "ac_build: out is NULL");
    *out = nullptr;
    ac_automaton *a = nullptr;
    try {
        a = new ac_automaton();
    } catch (...) {
        return set_error(AC_ENOMEM, "ac_build: host allocation");
    }
    a->placement = opts ? opts->placement : AC_PLACE_AUTO;
    a->machine = opts ? opts->machine : AC_MACHINE_DFA;
    if (a->machine != AC_MACHINE_DFA && a->machine != AC_MACHINE_PFAC) {
        delete a;
        return set_error(AC_EINVAL, "ac_build: unknown machine kind %d", opts->machine);
    }
    a->device = opts ? opts->device : 0;
    a->smem_cap_bytes = opts ? opts->smem_table_bytes : 0;
    if (a->placement < AC_PLACE_AUTO || a->placement > AC_PLACE_HYBRID16) {
        const int placement = a->placement;
        delete a;
        return set_error(AC_EINVAL, "ac_build: unknown placement %d", placement);
    }
    int rc;
    try {
        rc = build_machines(pats, lens, P, opts, a);
    } catch (const std::bad_alloc &) {
        rc = set_error(AC_ENOMEM, "ac_build: host allocation");
    }
    if (rc == AC_OK && a->sigma == 4)
        for (auto &s : a->subs)
            if (s.states >= (1u << 30)) rc = set_error(AC_ERANGE, "ac_build: 2^30 states or more");
    if (rc == AC_OK && a->device >= 0) {
        rc = upload(a);
        if (rc == AC_OK) rc = check_smem_placement(a);
    }
    if (rc != AC_OK) {
        free_device(a);
        delete a;
        return rc;
    }
    if (log_level() >= 2) {
        uint64_t states = 0;
        for (auto &sb : a->subs) states += sb.states;
        ac_log(2, "build: %u patterns, %u subsets, alphabet of %u, %llu states, %.2f ms build, %.2f ms upload",
               a->P, a->K, a->sigma, (unsigned long long)states, a->build_ms, a->upload_ms);
    }
    *out = a;
    return AC_OK;
}

void ac_free(ac_automaton *a) {
    if (!a) return;
    free_device(a);
    delete a;
}

}  // extern "C"

// ------------------------------------------------------------------ save / load
// File layout (host byte order; written and read by this library only):
// magic, format version, the automaton's fields, then per subset its
// scalars and its tables, each table as a 64-bit element count followed by
// the elements. The scan configuration is not kept (a loaded automaton starts
// at the defaults); nothing device-side is written.
namespace {
constexpr char kFileMagic[8] = {'A', 'C', 'G', 'B', '3', '0', '0', 'M'};
constexpr uint32_t kFileFormat = 1;

struct FileWriter {
    FILE *f;
    bool ok = true;
    template <class T>
    void put(const T &v) {
        ok = ok && fwrite(&v, sizeof(T), 1, f) == 1;
    }
    template <class T>
    void vec(const std::vector<T> &v) {
        const uint64_t n = v.size();
        put(n);
        if (n) ok = ok && fwrite(v.data(), sizeof(T), n, f) == n;
    }
};

struct FileReader {
    FILE *f;
    uint64_t left;  // bytes not yet read: bounds every count taken from the file
    bool ok = true;
    template <class T>
    void get(T &v) {
        ok = ok && left >= sizeof(T) && fread(&v, sizeof(T), 1, f) == 1;
        if (ok) left -= sizeof(T);
    }
    template <class T>
    void vec(std::vector<T> &v) {
        uint64_t n = 0;
        get(n);
        if (!ok || n > left / sizeof(T)) {
            ok = false;
            return;
        }
        v.resize(n);
        if (n) ok = fread(v.data(), sizeof(T), n, f) == n;
        if (ok) left -= n * sizeof(T);
    }
};

// Every index a scan would follow stays inside its table: a file that fails
// these checks is refused rather than handed to the kernels.
const char *check_loaded(const ac_automaton *a) {
    if (a->sigma == 0 || a->sigma > 255 || a->K == 0 || a->K > a->P || a->subs.size() != a->K)
        return "bad alphabet size or subset count";
    if (a->machine != AC_MACHINE_DFA && a->machine != AC_MACHINE_PFAC) return "unknown machine";
    uint32_t mapped = 0;
    for (int b = 0; b < 256; ++b) {
        if (a->sym_of_byte[b] > a->sigma) return "bad symbol map";
        if (a->sym_of_byte[b] < a->sigma) ++mapped;
    }
    // every symbol has exactly one byte, and byte_of_sym is the inverse map
    if (mapped != a->sigma) return "the symbol map does not give every symbol exactly one byte";
    for (uint32_t c = 0; c < a->sigma; ++c)
        if (a->sym_of_byte[a->byte_of_sym[c]] != c) return "byte_of_sym does not invert the symbol map";
    // the kernels decode A, C, G, T bytes by a fixed code when this flag is set
    const bool acgt = a->sigma == 4 && a->byte_of_sym[0] == 'A' && a->byte_of_sym[1] == 'C' &&
                      a->byte_of_sym[2] == 'G' && a->byte_of_sym[3] == 'T';
    if (acgt != a->dna_acgt) return "the ACGT flag disagrees with the alphabet";
    uint32_t next_id = 0, max_len = 0;
    for (const HostSubset &h : a->subs) {
        const uint64_t S = h.states;
        if (S == 0 || S >= (1u << 30)) return "bad state count";
        if (h.id_lo != next_id || h.id_hi <= h.id_lo || h.id_hi > a->P) return "bad pattern id ranges";
        next_id = h.id_hi;
        max_len = std::max(max_len, h.max_len);
        if (h.table.size() != S * a->sigma || h.out_off.size() != S + 1) return "table sizes disagree";
        if ((!h.fail.empty() && h.fail.size() != S) || (!h.depth.empty() && h.depth.size() != S))
            return "table sizes disagree";
        const bool pfac = a->machine == AC_MACHINE_PFAC;
        for (uint32_t e : h.table)
            if ((e & kStateMask) >= S && !(pfac && e == kMissing)) return "a transition leaves the machine";
        for (uint32_t f : h.fail)
            if (f >= S) return "a failure link leaves the machine";
        if (h.out_off[0] != 0 || h.out_off[S] != h.out_ids.size()) return "bad output offsets";
        for (uint64_t s = 0; s < S; ++s)
            if (h.out_off[s] > h.out_off[s + 1]) return "bad output offsets";
        for (uint32_t id : h.out_ids)
            if (id < h.id_lo || id >= h.id_hi) return "an output id outside the subset";
        if (!h.table2.empty()) {
            if (a->sigma != 4 || h.table2.size() != S * 16) return "bad two-symbol table";
            for (uint32_t e : h.table2)
                if ((e & kStateMask2) >= S) return "bad two-symbol table";
        }
        if (h.table16.size() != (uint64_t)h.rows16 * 4 || h.rows16 > S) return "bad 16-bit prefix";
        for (uint16_t e : h.table16)
            if ((uint64_t)(e >> 1) >= S) return "bad 16-bit prefix";
        if (h.table_e16.size() != (uint64_t)h.rows_e16 * 4 || h.rows_e16 > S) return "bad escape-coded prefix";
        for (uint16_t e : h.table_e16)
            if (e != kEsc16 && e >= S) return "bad escape-coded prefix";
        if ((!h.table16.empty() || !h.table_e16.empty()) && a->sigma != 4) return "16-bit prefix for a 4-letter machine only";
    }
    if (next_id != a->P || max_len != a->max_len) return "pattern ids or lengths disagree";
    return nullptr;
}
}  // namespace

extern "C" {

int ac_save(const ac_automaton *a, const char *path) {
    if (!a || !path) return set_error(AC_EINVAL, "ac_save: NULL argument");
    FILE *f = fopen(path, "wb");
    if (!f) return set_error(AC_EINVAL, "ac_save: cannot open %s for writing", path);
    FileWriter w{f};
    for (char c : kFileMagic) w.put(c);
    w.put(kFileFormat);
    w.put(a->P);
    w.put(a->K);
    w.put(a->sigma);
    w.put(a->max_len);
    w.put(a->placement);
    w.put(a->machine);
    w.put(a->smem_cap_bytes);
    w.put((uint8_t)a->dna_acgt);
    w.put((uint8_t)a->has_table2);
    for (int b = 0; b < 256; ++b) w.put(a->sym_of_byte[b]);
    for (int b = 0; b < 256; ++b) w.put(a->byte_of_sym[b]);
    w.put(a->build_ms);
    for (const HostSubset &h : a->subs) {
        w.put(h.id_lo);
        w.put(h.id_hi);
        w.put(h.max_len);
        w.put(h.states);
        w.put(h.rows16);
        w.put(h.rows_e16);
        for (double t : h.tail_mass) w.put(t);
        w.vec(h.table);
        w.vec(h.fail);
        w.vec(h.depth);
        w.vec(h.out_off);
        w.vec(h.out_ids);
        w.vec(h.table2);
        w.vec(h.table16);
        w.vec(h.table_e16);
    }
    const bool ok = w.ok && fflush(f) == 0;
    if (fclose(f) != 0 || !ok) return set_error(AC_EINVAL, "ac_save: write to %s failed", path);
    return AC_OK;
}

int ac_load(const char *path, int device, ac_automaton **out) {
    NvtxRange nvtx_range("ac_load");
    if (!path || !out) return set_error(AC_EINVAL, "ac_load: NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return set_error(AC_EINVAL, "ac_load: cannot open %s", path);
    uint64_t size = 0;
    if (fseek(f, 0, SEEK_END) == 0) {
        const long e = ftell(f);
        size = e > 0 ? (uint64_t)e : 0;
    }
    fseek(f, 0, SEEK_SET);
    ac_automaton *a = new (std::nothrow) ac_automaton();
    if (!a) {
        fclose(f);
        return set_error(AC_ENOMEM, "ac_load: host allocation");
    }
    int rc = AC_OK;
    try {
        FileReader r{f, size};
        char magic[8] = {};
        uint32_t format = 0;
        for (char &c : magic) r.get(c);
        r.get(format);
        if (!r.ok || memcmp(magic, kFileMagic, 8) != 0 || format != kFileFormat) {
            rc = set_error(AC_EINVAL, "ac_load: %s is not an automaton file of this library", path);
        } else {
            uint8_t acgt = 0, t2 = 0;
            r.get(a->P);
            r.get(a->K);
            r.get(a->sigma);
            r.get(a->max_len);
            r.get(a->placement);
            r.get(a->machine);
            r.get(a->smem_cap_bytes);
            r.get(acgt);
            r.get(t2);
            a->dna_acgt = acgt != 0;
            a->has_table2 = t2 != 0;
            for (int b = 0; b < 256; ++b) r.get(a->sym_of_byte[b]);
            for (int b = 0; b < 256; ++b) r.get(a->byte_of_sym[b]);
            r.get(a->build_ms);
            if (r.ok && (a->K == 0 || a->K > a->P)) r.ok = false;
            if (r.ok) a->subs.resize(a->K);
            for (uint32_t k = 0; r.ok && k < a->K; ++k) {
                HostSubset &h = a->subs[k];
                r.get(h.id_lo);
                r.get(h.id_hi);
                r.get(h.max_len);
                r.get(h.states);
                r.get(h.rows16);
                r.get(h.rows_e16);
                for (double &t : h.tail_mass) r.get(t);
                r.vec(h.table);
                r.vec(h.fail);
                r.vec(h.depth);
                r.vec(h.out_off);
                r.vec(h.out_ids);
                r.vec(h.table2);
                r.vec(h.table16);
                r.vec(h.table_e16);
            }
            if (!r.ok || r.left != 0) {
                rc = set_error(AC_EINVAL, "ac_load: %s is truncated or has trailing bytes", path);
            } else if (const char *why = check_loaded(a)) {
                rc = set_error(AC_EINVAL, "ac_load: %s: %s", path, why);
            }
        }
    } catch (const std::bad_alloc &) {
        rc = set_error(AC_ENOMEM, "ac_load: host allocation");
    }
    fclose(f);
    if (rc == AC_OK) {
        a->device = device;
        if (device >= 0) {
            rc = upload(a);
            if (rc == AC_OK) rc = check_smem_placement(a);
        }
    }
    if (rc != AC_OK) {
        free_device(a);
        delete a;
        return rc;
    }
    *out = a;
    return AC_OK;
}

int ac_stats(const ac_automaton *a, ac_stats_t *o) {
    if (!a || !o) return set_error(AC_EINVAL, "ac_stats: NULL argument");
    memset(o, 0, sizeof(*o));
    o->num_patterns = a->P;
    o->num_subsets = a->K;
    o->sigma = a->sigma;
    o->max_len = a->max_len;
    // the plan a scan of a long byte text (1 GiB) with the current configuration would use
    ScanPlan plan{};
    bool planned = false;
    if (a->device >= 0 && a->machine == AC_MACHINE_DFA) {
        ac_scan_config c{};
        default_config(a, 1ull << 30, AC_U8, &c);
        planned = plan_scan(a, c, AC_U8, &plan) == AC_OK;
    }
    // kernel modes of the plan: 0 all rows, 1 hybrid, 2 optimistic prefix, 3 16-bit prefix
    static const int32_t kPlacementOfMode[4] = {AC_PLACE_SMEM, AC_PLACE_HYBRID, AC_PLACE_OPT, AC_PLACE_HYBRID16};
    o->scan_placement = !planned ? -1
                        : plan.short_text ? (plan.mode == kShortFull ? AC_PLACE_SMEM : AC_PLACE_HYBRID16)
                        : plan.lean ? (plan.mode == kLeanSmem32 ? AC_PLACE_SMEM : AC_PLACE_HYBRID16)
                                    : kPlacementOfMode[plan.mode & 3];
    o->scan_stride = planned ? plan.stride : 0;
    o->scan_kernel = !planned ? -1 : plan.short_text ? AC_KERNEL_SHORT : plan.lean ? AC_KERNEL_LEAN : AC_KERNEL_GENERAL;
    for (auto &s : a->subs) {
        o->states += s.states;
        o->table_bytes += (uint64_t)s.table.size() * 4;
        o->output_entries += s.out_ids.size();
        o->table2_bytes += (uint64_t)s.table2.size() * 4;
        if (planned && plan.short_text)
            o->smem_states += std::min<uint64_t>(plan.mode == kShortFull ? s.states : s.rows_e16, plan.smem_rows);
        else if (planned && plan.lean)
            o->smem_states += std::min<uint64_t>(plan.mode == kLeanSmem32 ? s.states : s.rows_e16,
                                                 plan.smem_rows);
        else if (planned)
            o->smem_states += std::min<uint64_t>(plan.mode == 3 ? s.rows16 : s.states, plan.smem_rows);
    }
    o->build_ms = a->build_ms;
    o->upload_ms = a->upload_ms;
    o->device = a->device;
    o->row_len = a->cfg.row_len;
    o->threads = a->cfg.threads;
    o->chains = a->cfg.chains;
    return AC_OK;
}

int ac_subset(const ac_automaton *a, uint32_t k, ac_subset_view *v) {
    if (!a || !v || k >= a->K) return set_error(AC_EINVAL, "ac_subset: bad argument");
    const HostSubset &s = a->subs[k];
    v->id_lo = s.id_lo;
    v->id_hi = s.id_hi;
    v->max_len = s.max_len;
    v->sigma = a->sigma;
    v->states = s.states;
    v->smem_states = 0;
    v->table = s.table.data();
    v->fail = s.fail.data();
    v->depth = s.depth.data();
    v->out_off = s.out_off.data();
    v->out_ids = s.out_ids.data();
    v->symbol_of_byte = a->sym_of_byte;
    v->table2 = s.table2.empty() ? nullptr : s.table2.data();
    v->table16 = s.table16.empty() ? nullptr : s.table16.data();
    v->rows16 = s.rows16;
    v->table_e16 = s.table_e16.empty() ? nullptr : s.table_e16.data();
    v->rows_e16 = s.rows_e16;
    return AC_OK;
}

int ac_set_scan_config(ac_automaton *a, const ac_scan_config *cfg) {
    if (!a || !cfg) return set_error(AC_EINVAL, "ac_set_scan_config: NULL argument");
    if (cfg->threads && (cfg->threads % 32 || cfg->threads > 1024))
        return set_error(AC_EINVAL, "ac_set_scan_config: threads must be a multiple of 32, at most 1024");
    if (cfg->chains && (cfg->chains > 4 || (cfg->chains == 3 && cfg->kernel != AC_KERNEL_LEAN)))
        return set_error(AC_EINVAL, "ac_set_scan_config: chains must be 1, 2 or 4 (3 with the lean kernel)");
    if (cfg->kernel > AC_KERNEL_SHORT) return set_error(AC_EINVAL, "ac_set_scan_config: unknown kernel %u", cfg->kernel);
    if (cfg->stage_bytes && cfg->stage_bytes != 16 && cfg->stage_bytes != 32)
        return set_error(AC_EINVAL, "ac_set_scan_config: stage bytes must be 16 or 32");
    if (cfg->stride > 2) return set_error(AC_EINVAL, "ac_set_scan_config: stride must be 0, 1 or 2");
    if (cfg->stride == 2 && !a->has_table2)
        return set_error(AC_EINVAL, "ac_set_scan_config: stride 2 needs the automaton's two-symbol table");
    a->cfg = *cfg;
    return AC_OK;
}

int ac_get_scan_config(const ac_automaton *a, ac_scan_config *cfg) {
    if (!a || !cfg) return set_error(AC_EINVAL, "ac_get_scan_config: NULL argument");
    *cfg = a->cfg;
    return AC_OK;
}

void ac_result_free(ac_result *r) {
    if (!r) return;
    free(r->matches);
    free(r->counts);
    memset(r, 0, sizeof(*r));
}

int ac_results_take(ac_result *outs, uint32_t n, ac_match *matches, uint64_t *moff, uint64_t *counts,
                    uint64_t *coff) {
    if (n && (!outs || !moff)) return set_error(AC_EINVAL, "ac_results_take: NULL argument");
    if (counts && !coff) return set_error(AC_EINVAL, "ac_results_take: NULL argument");
    uint64_t mtot = 0;
    for (uint32_t i = 0; i < n; ++i) mtot += outs[i].num_matches;
    if (mtot && !matches) return set_error(AC_EINVAL, "ac_results_take: NULL argument");
    uint64_t m = 0, c = 0;
    if (n == 0) {
        if (moff) moff[0] = 0;
        if (coff) coff[0] = 0;
    }
    for (uint32_t i = 0; i < n; ++i) {
        ac_result &r = outs[i];
        moff[i] = m;
        if (r.num_matches) memcpy(matches + m, r.matches, r.num_matches * sizeof(ac_match));
        m += r.num_matches;
        if (counts) {
            coff[i] = c;
            if (r.counts) memcpy(counts + c, r.counts, (size_t)r.num_patterns * 8);
            else memset(counts + c, 0, (size_t)r.num_patterns * 8);
            c += r.num_patterns;
        }
        ac_result_free(&r);
    }
    if (n) {
        moff[n] = m;
        if (counts) coff[n] = c;
    }
    return AC_OK;
}

int ac_scan(const ac_automaton *a, const uint8_t *text, uint64_t n, int fmt, int mem, void *stream,
            ac_result *out) {
    NvtxRange nvtx_range("ac_scan");
    if (!out) return set_error(AC_EINVAL, "ac_scan: out is NULL");
    memset(out, 0, sizeof(*out));
    int rc = check_scan_args(a, n, fmt);
    if (rc) return rc;
    if (mem != AC_HOST && mem != AC_DEVICE) return set_error(AC_EINVAL, "ac_scan: unknown memory kind %d", mem);
    if (!text && n) return set_error(AC_EINVAL, "ac_scan: text is NULL");
    ac_result r{};
    r.num_patterns = a->P;
    r.counts = (uint64_t *)calloc(a->P, sizeof(uint64_t));
    if (!r.counts) return set_error(AC_ENOMEM, "ac_scan: host counts");
    if (n == 0) {
        *out = r;
        return AC_OK;
    }
    DeviceGuard g(a->device);
    if (!g.ok) {
        ac_result_free(&r);
        return set_error(AC_ECUDA, "ac_scan: cannot use device %d", a->device);
    }
    cudaStream_t s = (cudaStream_t)stream;
    rc = [&]() -> int {
        Scratch sc(s);
        const uint64_t nbytes = text_bytes(n, fmt);
        const uint8_t *d_text = nullptr;
        uint64_t readable = 0;
        // a large host text is copied in pieces while the pieces already on
        // the device are scanned (the host link, not the scan, sets the pace)
        const bool pipe = mem == AC_HOST && a->machine == AC_MACHINE_DFA && nbytes >= kPipeMinBytes;
        int e = AC_OK;
        if (pipe) {
            uint8_t *buf = (uint8_t *)sc.get((nbytes + 15) & ~15ull);
            if (!buf) return set_error(AC_ENOMEM, "scan: device text buffer of %llu bytes", (unsigned long long)nbytes);
            d_text = buf;
            readable = nbytes;
        } else {
            e = stage_text(text, nbytes, mem, s, sc, &d_text, &readable);
            if (e) return e;
        }
        // counter, error word, counts
        unsigned long long *num = (unsigned long long *)sc.get(16 + (size_t)a->P * 8);
        if (!num) return set_error(AC_ENOMEM, "ac_scan: scratch");
        uint32_t *err = (uint32_t *)(num + 1);
        unsigned long long *d_counts = num + 2;
        uint64_t cap = std::min<uint64_t>(n / 256 + 4096, 1ull << 26);
        ac_scan_config cfg;
        default_config(a, n, fmt, &cfg);
        if (pipe && !a->cfg.row_len && cfg.kernel != AC_KERNEL_SHORT) {
            // short rows, so that every piece spreads over all the SMs
            const uint64_t warm = fmt == AC_U8 ? a->max_len : (a->max_len + 3) / 4;
            const uint64_t rb = std::max<uint64_t>(128, 2 * ((warm + 31) / 32 * 32));
            cfg.row_len = (uint32_t)std::min<uint64_t>(rb * (fmt == AC_U8 ? 1 : 4), 1u << 20);
        }
        log_plan(a, n, fmt, cfg);
        // the lean kernel hands stages with matches to a second kernel (not in the piecewise scan)
        EmitEntry *q = nullptr;
        uint64_t q_cap = 0;
        if (!pipe && a->machine == AC_MACHINE_DFA && cfg.kernel == AC_KERNEL_LEAN) {
            q_cap = emit_queue_cap(n, fmt);
            q = (EmitEntry *)sc.get(q_cap * sizeof(EmitEntry));
        }
        unsigned long long h_num[2];
        unsigned long long *keys = nullptr;
        for (int attempt = 0; attempt < 2; ++attempt) {
            keys = (unsigned long long *)sc.get(cap * 8);
            if (!keys) return set_error(AC_ENOMEM, "ac_scan: %llu output slots", (unsigned long long)cap);
            CK(cudaMemsetAsync(num, 0, 16 + (size_t)a->P * 8, s), "ac_scan: memset");
            ScanText t{d_text, n, fmt, readable};
            ScanOut o{keys, cap, num, d_counts, err};
            if (q) {
                o.q = q;
                o.q_cap = q_cap;
            }
            if (pipe && attempt == 0)
                e = pipelined_scan(a, text, d_text, t, o, cfg, s);
            else
                e = launch_scan(a, t, o, cfg, s);
            if (e) return e;
            CK(cudaMemcpyAsync(h_num, num, 16, cudaMemcpyDeviceToHost, s), "ac_scan: copy count");
            CK(cudaStreamSynchronize(s), "ac_scan: scan");
            if ((uint32_t)h_num[1]) return set_error(AC_ETIMEDOUT, "ac_scan: a device-side wait ran out");
            if (h_num[0] <= cap) break;
            sc.release(keys);
            keys = nullptr;
            cap = h_num[0];
        }
        if (!keys) return set_error(AC_ERANGE, "ac_scan: output beyond capacity after a retry");
        const uint64_t M = h_num[0];
        if (M && M <= kSmallSortMax) {
            ac_match *d_m = (ac_match *)sc.get(M * sizeof(ac_match));
            if (!d_m) return set_error(AC_ENOMEM, "ac_scan: records");
            e = launch_small_sort(keys, num, M, (uint32_t)key_shift_for(a), d_m, nullptr, nullptr, s);
            if (e) return e;
            r.matches = (ac_match *)malloc(M * sizeof(ac_match));
            if (!r.matches) return set_error(AC_ENOMEM, "ac_scan: host matches");
            CK(cudaMemcpyAsync(r.matches, d_m, M * sizeof(ac_match), cudaMemcpyDeviceToHost, s),
               "ac_scan: copy matches");
        } else if (M) {
            unsigned long long *alt = (unsigned long long *)sc.get(M * 8);
            if (!alt) return set_error(AC_ENOMEM, "ac_scan: sort buffer");
            const int end_bit = (int)std::min<uint32_t>(64, key_shift_for(a) + bits_for(n - 1));
            size_t tb = 0;
            e = sort_keys(keys, alt, M, sort_begin_bit(a), end_bit, nullptr, &tb, s, nullptr);
            if (e) return e;
            void *temp = sc.get(tb);
            if (!temp) return set_error(AC_ENOMEM, "ac_scan: sort scratch");
            unsigned long long *sorted = nullptr;
            e = sort_keys(keys, alt, M, sort_begin_bit(a), end_bit, temp, &tb, s, &sorted);
            if (e) return e;
            ac_match *d_m = (ac_match *)(sorted == keys ? (void *)alt : (void *)keys);
            e = launch_keys_to_matches(sorted, num, M, (uint32_t)key_shift_for(a), d_m, nullptr, nullptr, s);
            if (e) return e;
            r.matches = (ac_match *)malloc(M * sizeof(ac_match));
            if (!r.matches) return set_error(AC_ENOMEM, "ac_scan: host matches");
            CK(cudaMemcpyAsync(r.matches, d_m, M * sizeof(ac_match), cudaMemcpyDeviceToHost, s),
               "ac_scan: copy matches");
        }
        CK(cudaMemcpyAsync(r.counts, d_counts, (size_t)a->P * 8, cudaMemcpyDeviceToHost, s), "ac_scan: copy counts");
        CK(cudaStreamSynchronize(s), "ac_scan: results");
        r.num_matches = M;
        return AC_OK;
    }();
    if (rc != AC_OK) {
        ac_result_free(&r);
        return rc;
    }
    *out = r;
    return AC_OK;
}

int ac_key_shift(const ac_automaton *a) { return a ? key_shift_for(a) : 0; }

// The scan up to unsorted keys. With err_out, the error word (or null when
// the kernel has no device-side waits) is handed to the caller, who reports
// it (the sort does); without, a marking kernel writes it into *d_num.
static int scan_keys(const ac_automaton *a, const uint8_t *d_text, uint64_t n, int fmt, cudaStream_t s, Scratch &sc,
                     uint64_t *d_keys, uint64_t cap, uint64_t *d_num, uint64_t *d_counts, const uint32_t **err_out) {
    int rc;
    const uint8_t *t = nullptr;
    uint64_t readable = 0;
    if (n) {
        rc = stage_text(d_text, text_bytes(n, fmt), AC_DEVICE, s, sc, &t, &readable);
        if (rc) return rc;
    }
    ac_scan_config cfg{};
    if (n) {
        default_config(a, n, fmt, &cfg);
        log_plan(a, n, fmt, cfg);
    }
    // the short-text kernel has no device-side waits: no error word to check
    const bool waits = n && !(a->machine == AC_MACHINE_DFA && cfg.kernel == AC_KERNEL_SHORT);
    // the lean kernel queues stages with matches and walks them after each row block
    const bool lean = waits && a->machine == AC_MACHINE_DFA && cfg.kernel == AC_KERNEL_LEAN;
    uint32_t *err = nullptr;
    EmitEntry *q = nullptr;
    uint64_t q_cap = 0;
    if (waits) {
        err = (uint32_t *)sc.get(16);
        if (!err) return set_error(AC_ENOMEM, "ac_scan_keys_async: scratch");
        if (lean) {
            q_cap = emit_queue_cap(n, fmt);
            q = (EmitEntry *)sc.get(q_cap * sizeof(EmitEntry));  // none: stages are walked again in place
        }
    }
    // error word, counter and counts zeroed by one launch
    // (overlapped: it waits for the launch before it, whatever that is, before writing)
    rc = launch_zero((unsigned long long *)err, err ? 2 : 0, (unsigned long long *)d_num, 1,
                     (unsigned long long *)d_counts, d_counts ? a->P : 0, s, true);
    if (rc) return rc;
    if (n) {
        ScanText tx{t, n, fmt, readable};
        ScanOut o{(unsigned long long *)d_keys, cap, (unsigned long long *)d_num, (unsigned long long *)d_counts,
                  err};
        o.after_zero = true;  // the zeroing launch is the one just before
        if (q) {
            o.q = q;
            o.q_cap = q_cap;
        }
        rc = launch_scan(a, tx, o, cfg, s);
        if (rc) return rc;
    }
    if (err_out) {
        *err_out = err;
        return AC_OK;
    }
    return waits ? launch_mark_error((unsigned long long *)d_num, err, s) : AC_OK;
}

int ac_scan_keys_async(const ac_automaton *a, const uint8_t *d_text, uint64_t n, int fmt, void *stream,
                       uint64_t *d_keys, uint64_t cap, uint64_t *d_num, uint64_t *d_counts) {
    NvtxRange nvtx_range("ac_scan_keys_async");
    int rc = check_scan_args(a, n, fmt);
    if (rc) return rc;
    if ((!d_text && n) || !d_num || (!d_keys && cap)) return set_error(AC_EINVAL, "ac_scan_keys_async: NULL argument");
    DeviceGuard g(a->device);
    if (!g.ok) return set_error(AC_ECUDA, "ac_scan_keys_async: cannot use device %d", a->device);
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    return scan_keys(a, d_text, n, fmt, s, sc, d_keys, cap, d_num, d_counts, nullptr);
}

// The sort of the keys into records; err (or null): a scan's error word,
// reported as *d_num_out = UINT64_MAX. overlap: the launch just before is
// this library's scan or zeroing, and the one-launch sort may start while it
// finishes (it waits for its writes).
static int sort_to_matches(const ac_automaton *a, uint64_t n, uint64_t *d_keys, const uint64_t *d_num, uint64_t cap,
                           cudaStream_t s, ac_match *d_matches, uint64_t *d_num_out, const uint32_t *err,
                           bool overlap = false) {
    if (cap <= kSmallSortMax)
        return launch_small_sort((const unsigned long long *)d_keys, (const unsigned long long *)d_num, cap,
                                 (uint32_t)key_shift_for(a), d_matches, (unsigned long long *)d_num_out, err, s,
                                 overlap);
    Scratch sc(s);
    const uint64_t kcap = cap ? cap : 1;
    unsigned long long *alt = (unsigned long long *)sc.get(kcap * 8);
    if (!alt) return set_error(AC_ENOMEM, "ac_sort_keys_async: scratch");
    int rc = AC_OK;
    unsigned long long *sorted = (unsigned long long *)d_keys;
    if (cap) {
        // entries [M, cap) become the largest key so they sort last
        rc = launch_pad_keys((unsigned long long *)d_keys, (const unsigned long long *)d_num, cap, s);
        if (rc) return rc;
        const int end_bit = (int)std::min<uint32_t>(64, key_shift_for(a) + bits_for(n ? n - 1 : 0));
        size_t tb = 0;
        rc = sort_keys((unsigned long long *)d_keys, alt, cap, sort_begin_bit(a), end_bit, nullptr, &tb, s, nullptr);
        if (rc) return rc;
        void *temp = sc.get(tb);
        if (!temp) return set_error(AC_ENOMEM, "ac_sort_keys_async: sort scratch");
        rc = sort_keys((unsigned long long *)d_keys, alt, cap, sort_begin_bit(a), end_bit, temp, &tb, s, &sorted);
        if (rc) return rc;
    }
    return launch_keys_to_matches(sorted, (const unsigned long long *)d_num, cap, (uint32_t)key_shift_for(a),
                                  d_matches, (unsigned long long *)d_num_out, err, s);
}

int ac_sort_keys_async(const ac_automaton *a, uint64_t n, uint64_t *d_keys, const uint64_t *d_num, uint64_t cap,
                       void *stream, ac_match *d_matches, uint64_t *d_num_out) {
    NvtxRange nvtx_range("ac_sort_keys_async");
    if (!a || !d_num || (cap && (!d_keys || !d_matches)))
        return set_error(AC_EINVAL, "ac_sort_keys_async: NULL argument");
    if (a->device < 0) return set_error(AC_EINVAL, "ac_sort_keys_async: host-only automaton");
    DeviceGuard g(a->device);
    if (!g.ok) return set_error(AC_ECUDA, "ac_sort_keys_async: cannot use device %d", a->device);
    return sort_to_matches(a, n, d_keys, d_num, cap, (cudaStream_t)stream, d_matches, d_num_out, nullptr);
}

int ac_scan_async(const ac_automaton *a, const uint8_t *d_text, uint64_t n, int fmt, void *stream,
                  ac_match *d_matches, uint64_t cap, uint64_t *d_num_matches, uint64_t *d_counts) {
    NvtxRange nvtx_range("ac_scan_async");
    int rc = check_scan_args(a, n, fmt);
    if (rc) return rc;
    if ((!d_text && n) || !d_num_matches || (!d_matches && cap))
        return set_error(AC_EINVAL, "ac_scan_async: NULL argument");
    DeviceGuard g(a->device);
    if (!g.ok) return set_error(AC_ECUDA, "ac_scan_async: cannot use device %d", a->device);
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc(s);
    uint64_t *keys = (uint64_t *)sc.get((cap ? cap : 1) * 8);
    if (!keys) return set_error(AC_ENOMEM, "ac_scan_async: scratch");
    // the sort reports the scan's error word (no separate marking launch)
    const uint32_t *err = nullptr;
    rc = scan_keys(a, d_text, n, fmt, s, sc, keys, cap, d_num_matches, d_counts, &err);
    if (rc) return rc;
    return sort_to_matches(a, n, keys, d_num_matches, cap, s, d_matches, d_num_matches, err, true);
}

}  // extern "C"
