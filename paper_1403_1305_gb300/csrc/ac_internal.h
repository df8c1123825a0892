// Internal declarations shared by the translation units of libacgb300.
#pragma once

#include <cuda_runtime.h>
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define AC_HAVE_NVTX 1
#endif
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ac.h"

namespace acgb {

constexpr uint32_t kFlag = 0x80000000u;  // table entry bit: next state has a non-empty output
constexpr uint32_t kStateMask = 0x7fffffffu;
constexpr uint32_t kMissing = 0x7fffffffu;  // failure-less table: no transition
// two-symbol table entries: bit 31 = output at the second symbol, bit 30 = at the first
constexpr uint32_t kFlag1 = 0x40000000u;
constexpr uint32_t kStateMask2 = 0x3fffffffu;
constexpr uint32_t kMaxStates2 = 1u << 28;  // s*16 + column must fit 32 bits
// escape-coded 16-bit prefix (lean scan): entry = next state, or kEsc16 when the
// next state has an output or does not fit 16 bits (read the 32-bit table)
constexpr uint32_t kEsc16 = 0xffffu;
constexpr uint32_t kRowsE16 = 1u << 15;  // rows built (256 KB): more than shared memory holds

// ---------------------------------------------------------------- host machine
struct HostSubset {
    uint32_t id_lo = 0, id_hi = 0;  // global pattern ids [id_lo, id_hi)
    uint32_t max_len = 0;
    uint32_t states = 0;
    std::vector<uint32_t> table;    // states * sigma, breadth-first ids | kFlag
    std::vector<uint32_t> fail;     // breadth-first ids
    std::vector<uint32_t> depth;
    std::vector<uint32_t> out_off;  // states + 1
    std::vector<uint32_t> out_ids;  // global ids, ascending per state
    std::vector<uint32_t> table2;   // sigma = 4 only: states * 16, two symbols per entry (or empty)
    // tail_mass[k] = sum over states s >= 2^k of the probability that an
    // i.i.d. text (letters drawn with the patterns' letter frequencies) ends
    // with s's string: an upper bound on the share of lookups at states >= 2^k
    double tail_mass[32] = {};
    // 16-bit prefix (sigma = 4): rows [0, rows16) whose next states all fit
    // 15 bits; entry = (next state << 1) | 1 when its output is not empty
    std::vector<uint16_t> table16;
    uint32_t rows16 = 0;
    // escape-coded 16-bit prefix (sigma = 4): rows [0, rows_e16), entry =
    // next state, or kEsc16 when that state has an output or is >= kEsc16
    std::vector<uint16_t> table_e16;
    uint32_t rows_e16 = 0;
};

// Device descriptor of one subset machine (array in device memory, one per subset).
struct SubsetDev {
    const uint32_t *table;    // states * sigma
    const uint32_t *table2;   // states * 16 (two-symbol table) or null
    const uint16_t *table16;  // rows16 * 4 (16-bit prefix) or null
    uint32_t rows16;
    const uint16_t *table_e16;  // rows_e16 * 4 (escape-coded 16-bit prefix) or null
    uint32_t rows_e16;
    const uint32_t *out_off;  // states + 1
    const uint32_t *out_ids;
    uint32_t states;
    uint32_t smem_states;     // rows [0, smem_states) are staged into shared memory
    uint32_t warm;            // max_len - 1: symbols of warm-up a chain needs
    uint32_t id_lo;
};

// One text of a batch, laid out from row `row_begin` of the arena.
struct BatchItemDev {
    uint64_t row_begin;  // first arena row
    uint64_t rows;       // rows it occupies
    uint64_t nsym;       // symbols
    uint64_t vbase;      // arena position of its first symbol (key position base)
    uint64_t cbase;      // offset of its counts in the counts array
};

struct BatchTileDev {
    uint32_t machine;    // index into the machine (subset) descriptors
    uint32_t pad;
    uint64_t row0;       // first arena row of the tile
};

struct DeviceSubset {
    uint32_t *table = nullptr, *out_off = nullptr, *out_ids = nullptr, *table2 = nullptr;
    uint16_t *table16 = nullptr, *table_e16 = nullptr;
};

}  // namespace acgb

struct ac_automaton {
    uint32_t P = 0, K = 1, sigma = 0, max_len = 0;
    uint8_t sym_of_byte[256];   // sigma = outside the alphabet
    uint8_t byte_of_sym[256];
    bool dna_acgt = false;      // alphabet is exactly "ACGT" in this order
    int32_t placement = AC_PLACE_AUTO;
    int32_t machine = AC_MACHINE_DFA;
    bool has_table2 = false;    // every subset has its two-symbol table
    int32_t device = -1;
    uint32_t smem_cap_bytes = 0;
    std::vector<acgb::HostSubset> subs;
    // device side
    std::vector<acgb::DeviceSubset> dsubs;
    acgb::SubsetDev *d_desc = nullptr;   // K descriptors
    std::vector<acgb::SubsetDev> h_desc; // host copy of the descriptors
    uint32_t table_smem_bytes = 0;       // bytes of table staged in shared memory per CTA (max over subsets)
    ac_scan_config cfg{};
    double build_ms = 0, upload_ms = 0;
};

namespace acgb {

// build.cpp
int build_machines(const uint8_t *const *pats, const uint32_t *lens, uint32_t P, const ac_build_opts *opts,
                   ac_automaton *a);
// gbuild.cu: subset [lo, hi) built on the current device (same machine as the host build)
int build_subset_device(const uint8_t *const *pats, const uint32_t *lens, uint32_t lo, uint32_t hi,
                        const uint8_t *sym_of_byte, uint32_t sigma, HostSubset &S, std::string &why);
// symbols per lookup a scan of this format uses under configuration stride `want` (0 = automatic)
uint32_t scan_stride(const ac_automaton *a, int fmt, uint32_t want);

// A named NVTX range over a host phase (a no-op unless a profiler records NVTX).
struct NvtxRange {
#ifdef AC_HAVE_NVTX
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
#else  // a toolkit without the NVTX headers: no ranges
    explicit NvtxRange(const char *) {}
#endif
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Limit (ns) of the bounded device-side waits of the next scan launch: 2 s,
// or 0 (the launch's first wait gives up) for the next N launches when the
// environment sets AC_FAULT_WAIT=N (read once; capi.cu).
uint64_t wait_limit_ns();

// error reporting and the AC_LOG diagnostics (capi.cu)
int set_error(int code, const char *fmt, ...);
int log_level();
void ac_log(int level, const char *fmt, ...);

// scan.cu
struct ScanText {
    const uint8_t *d_text;  // 16-byte aligned device pointer
    uint64_t n;             // symbols
    int fmt;
    uint64_t readable;      // bytes that may be read at d_text (>= the text's bytes; 0 = exactly those)
    // rows [row_begin, row_end) of the text's row geometry only (row_end 0 = to the last row): a text
    // scanned in pieces as it arrives, with the same row length in every launch
    uint64_t row_begin = 0, row_end = 0;
};

// A stage of text whose walk is right but whose matches are still to be
// emitted: the lean kernel walks such stages again, with their emission,
// once the warp's row block is done instead of in the middle of it.
struct EmitEntry {
    uint32_t row;    // text row (0xffffffff: none)
    uint32_t stage;  // stage index within the row's walk (warm-up stages first)
    uint32_t s;      // state before the stage
    uint32_t pad;
};

struct ScanOut {
    unsigned long long *keys;   // (pos << 32 | id), capacity `cap`
    uint64_t cap;
    unsigned long long *num;    // match counter (device)
    unsigned long long *counts; // per-pattern counts (device) or null
    uint32_t *err;              // device error word
    // optional scratch of q_cap queue entries (lean kernel), split evenly between the launch's warps;
    // null: stages with matches are walked again in place
    EmitEntry *q = nullptr;
    uint64_t q_cap = 0;
    // the scan kernel may start while the launch before it in the stream (the
    // zeroing of num and counts) still runs; it waits for that launch's
    // writes before its own first write to num, counts or keys
    bool after_zero = false;
};

// Stage geometry shared by host planning and the kernels.
constexpr uint32_t kStageBytes = 32;   // bytes of one chain's text per pipeline stage
// Short-text kernel: rows of at most 64 bytes (by default about kShortRows
// rows); the automatic choice takes it for texts of up to kShortAutoSymbols
// symbols; its table room keeps two CTAs per SM.
constexpr uint32_t kShortMaxRowBytes = 64;
constexpr uint64_t kShortRows = 150000;
constexpr uint64_t kShortAutoSymbols = 8ull << 20;
constexpr uint32_t kShortSmemBytes = 96u << 10;
uint32_t short_row_bytes(const ac_scan_config &cfg, int fmt);
const char *short_unfit(const ac_automaton *a, const ac_scan_config &c, int fmt);

int scan_smem_limit(int device);
uint64_t scan_row_bytes(const ac_scan_config &cfg, int fmt, uint64_t readable);
uint32_t scan_stage_bytes_per_cta(const ac_scan_config &cfg);
void default_config(const ac_automaton *a, uint64_t n, int fmt, ac_scan_config *cfg);
int launch_scan(const ac_automaton *a, const ScanText &t, const ScanOut &o, const ac_scan_config &cfg,
                cudaStream_t stream);
// entries of the lean kernel's emission queue for a text of n symbols (capi.cu)
uint64_t emit_queue_cap(uint64_t n, int fmt);
// Table placement and symbols per lookup of a single-text scan (format fmt)
// under configuration cfg (defaults filled in): kernel mode (the kernels'
// MODE_* values), table rows staged in shared memory, words of shared memory
// for the table, dynamic shared memory bytes.
// table placements of the lean kernel (ScanPlan::mode when ScanPlan::lean)
enum { kLeanSmem32 = 0, kLeanE16 = 1 };
// table placements of the short-text kernel (ScanPlan::mode when ScanPlan::short_text)
enum { kShortFull = 0, kShortE16 = 1 };
struct ScanPlan {
    bool lean = false;  // the lean kernel (mode = kLeanSmem32 or kLeanE16)
    bool short_text = false;  // the short-text kernel (mode = kShortFull or kShortE16)
    int mode = 0;
    uint32_t stride = 1;
    uint32_t smem_rows = 0;
    uint32_t table_words = 0;
    size_t smem = 0;
};
int plan_scan(const ac_automaton *a, const ac_scan_config &cfg, int fmt, ScanPlan *out);
// failure-less machine: one walk per start position (pfac.cu)
int launch_pfac(const ac_automaton *a, const ScanText &t, const ScanOut &o, const ac_scan_config &cfg,
                cudaStream_t stream);

// Several texts laid out in one arena of whole rows (ac_scan_batch, serving).
struct BatchLaunch {
    const uint8_t *arena;        // 16-byte aligned; rows * row_bytes bytes readable
    uint64_t rows;
    uint32_t row_bytes;          // multiple of kStageBytes
    int fmt;
    const BatchItemDev *items;   // device, sorted by row_begin
    uint32_t num_items;
    const BatchTileDev *tiles;   // device
    uint64_t num_tiles;
    const SubsetDev *machines;   // device, one per (automaton, subset)
    uint32_t max_states;         // over the machines
    uint32_t sigma;              // common to every automaton of the launch
    const uint8_t *sym_of_byte;  // 256 entries, common
    bool acgt;
    uint32_t key_shift;
    int placement;
    uint32_t smem_cap_bytes;
    int device;
    ac_scan_config cfg;          // threads and chains (row length is row_bytes)
    uint32_t track_flags;        // record flagged steps in the fast loop
};
int launch_scan_batch(const BatchLaunch &b, const ScanOut &o, cudaStream_t stream);
// shared-memory plan of a launch: table rows held in shared memory and the dynamic size
int plan_smem(int device, const ac_scan_config &cfg, uint32_t sigma, int placement, uint32_t smem_cap,
              uint32_t max_states, uint32_t *rows_used, bool *hybrid, size_t *smem_bytes, uint32_t *table_words);
int launch_fill_u64(unsigned long long *p, uint64_t count, unsigned long long value, cudaStream_t stream);
// zero three ranges of 8-byte words (a pointer may be null when its count is 0) in one launch;
// overlap: it may start while the launch before it in the stream still runs (it waits for that
// launch before writing; a scan launched overlapped behind it reads nothing written before the
// call until it has finished)
int launch_zero(unsigned long long *p0, uint64_t n0, unsigned long long *p1, uint64_t n1, unsigned long long *p2,
                uint64_t n2, cudaStream_t stream, bool overlap = false);
int launch_keys_to_matches(const unsigned long long *keys, const unsigned long long *num, uint64_t cap,
                           uint32_t shift, ac_match *out, unsigned long long *num_out, const uint32_t *err,
                           cudaStream_t stream);
int key_shift_for(const ac_automaton *a);
int launch_pad_keys(unsigned long long *keys, const unsigned long long *num, uint64_t cap, cudaStream_t stream);
int launch_mark_error(unsigned long long *num, const uint32_t *err, cudaStream_t stream);
// One-time process state of the scan launches (the tensor-map encoder, the
// rank sort's shared-memory attribute), set up before a first call that may
// run under stream capture.
void prime_scan_state();

// single-launch sort + record conversion of the first min(*num, cap) keys, cap at most kSmallSortMax
constexpr uint64_t kSmallSortMax = 8192;
// overlap: the sort may start while the launch before it in the stream (one
// of this library's scan or zeroing kernels) still runs; it waits for that
// launch's writes before reading anything
int launch_small_sort(const unsigned long long *keys, const unsigned long long *num, uint64_t cap, uint32_t shift,
                      ac_match *out, unsigned long long *num_out, const uint32_t *err, cudaStream_t stream,
                      bool overlap = false);
int sort_keys(unsigned long long *keys, unsigned long long *keys_alt, uint64_t count, int begin_bit, int end_bit,
              void *temp, size_t *temp_bytes, cudaStream_t stream, unsigned long long **sorted);
// first key bit a sort of a's keys must look at (stable sorts)
int sort_begin_bit(const ac_automaton *a);

// memory (capi.cu)
void *dev_alloc(size_t bytes, cudaStream_t stream);
void dev_free(void *p, cudaStream_t stream);

}  // namespace acgb
