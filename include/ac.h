/*
 * ac.h — C ABI of libacgb300: exact multiple-pattern matching (Aho-Corasick)
 * with the scan on an NVIDIA GB300 (sm_103a).
 *
 * Problem (paper, Abstract and Section I): locate every occurrence of a set
 * of patterns in a text. The result of a scan is the set
 *     M = { (e, j) : |P_j| <= e+1 <= n  and  text[e-|P_j|+1 .. e] = P_j }
 * as ac_match records sorted by end position e (0-based, inclusive), then by
 * pattern id j (the index of P_j in the array given to ac_build), and
 * counts[j] = the number of records with pattern id j.
 *
 * The machine (Section II.A): goto function, failure function and output
 * function, with failure transitions folded into regular ones (the "AC-opt"
 * machine of Section III, reference [4]) so the scan does one table lookup
 * per text symbol. Two partition axes (Section III): the text is cut into
 * chunks, each warmed up on the (longest pattern - 1) symbols before it
 * (input-focused split), and the pattern set can be cut into K subsets with
 * one machine each, all scanning the same text (pattern-focused split, the
 * paper's Fig. 5 approach).
 *
 * Conventions for every call:
 *  - Return value: AC_OK (0) or a negative AC_E* code; on error no output is
 *    produced (result structs are left zeroed) and ac_last_error() returns a
 *    one-line description for the calling thread.
 *  - Diagnostics: the environment variable AC_LOG (read once) set to 1
 *    prints every error message on stderr; 2 also prints one line per build
 *    (patterns, subsets, states, times), per scan plan (kernel, row length,
 *    CTA shape) and per batch path. The library marks its host phases with
 *    NVTX ranges (build, scan, sort, copies) for profilers that record them.
 *  - Pointers marked "device" are CUDA device pointers on the automaton's
 *    device; "host" pointers are ordinary (pageable or pinned) host memory.
 *  - Inputs are borrowed for the duration of the call only (asynchronous
 *    calls: until the work queued on the stream has finished).
 *  - Objects returned through ac_automaton**, ac_server** and ac_result are
 *    owned by the library; release them with ac_free, ac_serve_destroy and
 *    ac_result_free.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).
 *  - One automaton may be used by several threads and streams at once; scans
 *    do not modify it (ac_tune and ac_set_scan_config do, and must not race
 *    with scans of the same automaton).
 */
#ifndef AC_H
#define AC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AC_API __attribute__((visibility("default")))
#else
#define AC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ return codes */
#define AC_OK 0
#define AC_EINVAL (-1)    /* bad argument: NULL, P = 0, empty pattern, byte outside the alphabet, bad fmt */
#define AC_ENOMEM (-2)    /* host or device allocation failed */
#define AC_ERANGE (-3)    /* size limit: n >= 2^32, too many states, output beyond capacity after a retry */
#define AC_ECUDA (-4)     /* a CUDA call failed (no device, launch error, ...) */
#define AC_ETIMEDOUT (-5) /* a bounded device-side wait ran out, or ac_serve_wait timed out */
#define AC_EAGAIN (-6)    /* result not ready yet (ac_serve_poll) */
#define AC_EBUSY (-7)     /* server queue full (non-blocking submit refused) */

/* ------------------------------------------------------------ enums */
#define AC_U8 0      /* one byte per symbol */
#define AC_PACKED2 1 /* 2-bit codes, 4 symbols per byte; symbol i at bits 2*(i%4) of byte i/4;
                        code k stands for the k-th letter of a 4-letter alphabet */

#define AC_HOST 0
#define AC_DEVICE 1

#define AC_PLACE_AUTO 0   /* pick per subset: whole table in shared memory if it fits, else hybrid */
#define AC_PLACE_SMEM 1   /* whole table in shared memory; AC_ERANGE at build if it does not fit */
#define AC_PLACE_HYBRID 2 /* the first (breadth-first) states in shared memory, the rest read through L2 */
#define AC_PLACE_GLOBAL 3 /* every lookup through L2 / HBM */
#define AC_PLACE_OPT 4    /* a power-of-two breadth-first prefix in shared memory, read without a per-lookup
                             placement check; a stage of text that reaches a state beyond it is walked again
                             (exact either way). AC_PLACE_AUTO picks it for a one-symbol scan when the states
                             beyond the prefix are rarely reached (estimated from the patterns' letter
                             frequencies); batched scans use AC_PLACE_HYBRID instead. */
#define AC_PLACE_HYBRID16 5 /* 4-letter alphabets: a breadth-first prefix of 16-bit entries (next state + output
                               bit, for the rows whose next states fit 15 bits: about twice the rows of
                               AC_PLACE_HYBRID) in shared memory, the rest read through L2. AC_PLACE_AUTO picks
                               it for a one-symbol scan when it leaves fewer lookups to L2; batched scans use
                               AC_PLACE_HYBRID instead. */

#define AC_MACHINE_DFA 0  /* failure transitions folded into a dense next-state table (Section III, AC-opt):
                             one lookup per text symbol */
#define AC_MACHINE_PFAC 1 /* failure-less machine (Section II.B, the paper's Section IV method): goto function
                             only, built without a failure function; the scan walks from every text
                             position until a missing transition */

/* ------------------------------------------------------------ types */
typedef struct ac_automaton ac_automaton;
typedef struct ac_server ac_server;

typedef struct {
    uint32_t pos;        /* 0-based end position (inclusive) of the occurrence */
    uint32_t pattern_id; /* index of the pattern in the array given to ac_build */
} ac_match;

typedef struct {
    const char *alphabet;  /* NUL-terminated string of distinct bytes forming the alphabet (order = symbol
                              codes, e.g. "ACGT"), or NULL: the distinct bytes of the patterns, ascending.
                              Text bytes outside it send the machine to the root state. */
    uint32_t num_subsets;  /* K >= 1 pattern-subset machines over contiguous id ranges of ceil(P/K);
                              0 means 1; K > P is AC_EINVAL */
    int32_t placement;     /* AC_PLACE_* */
    int32_t device;        /* CUDA device ordinal; -1 builds on the host only (inspection, no scans) */
    uint32_t smem_table_bytes; /* cap on table bytes held in shared memory per CTA; 0 = as much as fits */
    int32_t machine;           /* AC_MACHINE_DFA (default) or AC_MACHINE_PFAC; the results are the same */
    uint32_t stride;           /* symbols per table lookup the DFA machine is built for: 0 = automatic (the
                                  two-symbol table too for a 4-letter alphabet whose subsets are small enough
                                  for a scan to choose it: most visits within the first ~2,048 states, as
                                  estimated from the patterns' letter frequencies), 1 = one-symbol table only,
                                  2 = always the two-symbol table too (4-letter alphabets and the DFA machine
                                  only, else AC_EINVAL). The two-symbol table composes two transitions of the
                                  one-symbol table (16 columns per state, 4x its memory) so a scan does one
                                  dependent lookup per two text symbols; results are the same. */
    uint32_t builder;          /* AC_BUILDER_HOST (default) or AC_BUILDER_DEVICE: where the goto, failure and
                                  output functions are constructed; the machine is the same, state for state */
} ac_build_opts;

/* Machine construction (ac_build_opts.builder). */
#define AC_BUILDER_HOST 0   /* host threads, one per subset */
#define AC_BUILDER_DEVICE 1 /* on the automaton's GPU (DFA machine, device >= 0; else AC_EINVAL): patterns
                               sorted by symbol string, the trie numbered breadth-first from the longest
                               common prefixes of neighbours in that order, failure function, fold and output
                               function one depth at a time; the tables are then copied to the host view */

typedef struct {
    ac_match *matches;     /* host array of num_matches records, sorted; library-owned */
    uint64_t num_matches;
    uint64_t *counts;      /* host array of num_patterns counts; library-owned */
    uint32_t num_patterns;
} ac_result;

typedef struct {
    uint32_t num_patterns;
    uint32_t num_subsets;
    uint32_t sigma;          /* alphabet size */
    uint32_t max_len;        /* longest pattern */
    uint64_t states;         /* sum over subsets */
    uint64_t table_bytes;    /* sum over subsets of the dense goto tables */
    uint64_t output_entries; /* sum over states of |output(state)| */
    uint64_t smem_states;    /* sum over subsets of the table rows a scan of byte text holds in shared memory */
    double build_ms;         /* host time of trie + failure + fold + renumber (all subsets) */
    double upload_ms;        /* host->device copy of the tables */
    int32_t device;
    uint32_t row_len;        /* current scan configuration (symbols per chain) */
    uint32_t threads;
    uint32_t chains;
    uint64_t table2_bytes;   /* sum over subsets of the two-symbol tables (0 if not built) */
    int32_t scan_placement;  /* the table placement (AC_PLACE_SMEM, _HYBRID, _OPT or _HYBRID16) and symbols per */
    uint32_t scan_stride;    /* lookup a scan of a long byte text (1 GiB; shorter texts may run the short-text
                                kernel) would use with the current configuration; -1 and 0
                                when not applicable (host-only automaton, failure-less machine) */
    int32_t scan_kernel;     /* AC_KERNEL_GENERAL, AC_KERNEL_LEAN or AC_KERNEL_SHORT: the kernel such a scan
                                runs (-1 when not applicable) */
} ac_stats_t;

/* Read-only host view of one subset machine (valid until ac_free). States are
 * numbered breadth-first (root 0). table[s*sigma + c] = next state of s on
 * symbol c, with bit 31 set when the next state's output is not empty.
 * out_ids[out_off[s] .. out_off[s+1]) = output(s), ascending global ids. */
typedef struct {
    uint32_t id_lo, id_hi;   /* pattern ids [id_lo, id_hi) of this subset */
    uint32_t max_len;        /* longest pattern of the subset */
    uint32_t sigma;
    uint32_t states;
    uint32_t smem_states;    /* states whose rows the scan keeps in shared memory */
    const uint32_t *table;   /* states x sigma */
    const uint32_t *fail;    /* states (failure function, breadth-first ids) */
    const uint32_t *depth;   /* states */
    const uint32_t *out_off; /* states + 1 */
    const uint32_t *out_ids;
    const uint8_t *symbol_of_byte; /* 256 entries; sigma = outside the alphabet */
    /* two-symbol table (NULL if not built): table2[s*16 + c1 + 4*c2] = the state after symbols c1 then c2
       from s (bits 0..29), bit 31 set when that state's output is not empty, bit 30 set when the output of
       the state after c1 alone is not empty */
    const uint32_t *table2;
    /* 16-bit prefix (4-letter alphabets; NULL otherwise): rows [0, rows16) are the longest breadth-first prefix
       whose next states all fit 15 bits; table16[s*4 + c] = (next << 1) | 1 if the next state's output is
       not empty */
    const uint16_t *table16;
    uint32_t rows16;
    /* escape-coded 16-bit prefix (4-letter alphabets, DFA machine; NULL otherwise), the lean kernel's shared-
       memory table: rows [0, rows_e16) (at most 32,768); table_e16[s*4 + c] = the next state when it is
       below 65,535 and its output is empty, else 65,535 (the lookup then reads table[]) */
    const uint16_t *table_e16;
    uint32_t rows_e16;
} ac_subset_view;

/* Scan configuration (ac_set_scan_config / ac_tune). Zero fields = defaults. */
typedef struct {
    uint32_t row_len;     /* text symbols per chain (rounded up to 32 bytes of text; to 16 bytes, at most 64,
                             for the short-text kernel) */
    uint32_t threads;     /* threads per CTA (multiple of 32; <= 512 for the general kernel; 512, 768 or
                             1024 for the lean one; 64 to 1024 for the short-text one) */
    uint32_t chains;      /* independent chains per thread: 1, 2 or 4 (3 too for the lean kernel; 1 for the
                             short-text kernel) */
    uint32_t ctas;        /* persistent grid size; 0 = one per SM */
    uint32_t stage_bytes; /* text bytes per chain per pipeline stage: 16 or 32 (16 needs 2 or 4 chains; the
                             lean kernel always uses 16) */
    uint32_t smem_table_bytes; /* cap on table bytes staged in shared memory for this scan (0 = the
                                  automaton's cap or as much as fits); a smaller table leaves more of the
                                  SM's memory to L1, which caches the rows a skewed text visits most */
    uint32_t stride;      /* symbols per lookup: 0 = automatic (2 when the automaton has its two-symbol
                             table and the text is ACGT bytes or packed, else 1), 1, or 2 (AC_EINVAL at scan
                             time when the two-symbol table or a suitable format is missing). Batched scans
                             use 1. */
    uint32_t kernel;      /* AC_KERNEL_*: which scan kernel a single-text scan runs (results are the same) */
} ac_scan_config;

/* Scan kernels (ac_scan_config.kernel). */
#define AC_KERNEL_AUTO 0    /* the short-text kernel for short texts where it applies, else the lean kernel
                               where it applies, else the general one */
#define AC_KERNEL_GENERAL 1 /* every table placement, alphabet and stride; threads <= 512, chains 1, 2 or 4 */
#define AC_KERNEL_LEAN 2    /* one-symbol scans of a 4-letter machine over ACGT bytes or packed text
                               (placement AUTO, SMEM or HYBRID16): the whole table in shared memory when it
                               fits, else an escape-coded 16-bit breadth-first prefix with the rest read
                               through L2; 16-byte stages; (threads, chains) in {(1024, 4), (1024, 3),
                               (1024, 2), (768, 4), (512, 4)}, default (1024, 2) for byte text and
                               (1024, 3) for packed text. AC_EINVAL at scan time when it does not apply. */
#define AC_KERNEL_SHORT 3   /* short texts on one 4-letter machine (one subset, any 4-letter alphabet, u8 or
                               packed text, placement AUTO, SMEM or HYBRID16): one thread per row of 16 to 64
                               bytes (row_len; by default about 150,000 rows: 16 bytes up to 2.4 MB of text,
                               longer rows above), its warm-up and row loaded straight into registers in one
                               round trip; the whole table in shared memory when it fits in 96 KB (all of the
                               SM's room with placement SMEM), else the escape-coded 16-bit prefix with the
                               rest read through L2. threads a multiple of 32 in [64, 1024] (default 512),
                               chains 1; the warm-up and the row at most nine 16-byte words. AC_KERNEL_AUTO
                               takes it for texts of at most 8 Mi symbols when the configuration is otherwise
                               untouched. AC_EINVAL at scan time when it does not apply. */

/* ------------------------------------------------------------ automaton */

/* Build the machines for patterns pats[0..P) (lengths lens[]), Section II.A
 * steps: goto function by inserting the patterns in order, failure function
 * breadth-first with output merge, failure transitions folded into a dense
 * table, states renumbered breadth-first; then (device >= 0) the tables are
 * copied to the device. Patterns are copied; the caller keeps ownership.
 * Errors: AC_EINVAL (pats/lens/out NULL, P = 0, an empty pattern, a byte
 * outside opts->alphabet, K > P), AC_ERANGE (>= 2^31 states in a subset, or
 * AC_PLACE_SMEM and a table that does not fit), AC_ENOMEM, AC_ECUDA. */
AC_API int ac_build(const uint8_t *const *pats, const uint32_t *lens, uint32_t P,
             const ac_build_opts *opts, ac_automaton **out);

/* Release an automaton (NULL is a no-op). */
AC_API void ac_free(ac_automaton *a);

/* Write automaton a (its machines, alphabet and build options; not its scan
 * configuration, nothing device-side) to the file at path, in this library's
 * own format (host byte order, versioned), so that ac_load can skip the
 * build. Errors: AC_EINVAL (NULL, the file cannot be written; ac_last_error
 * says which). */
AC_API int ac_save(const ac_automaton *a, const char *path);

/* Read an automaton written by ac_save and copy its tables to device
 * `device` (-1: host only, as ac_build with device -1). The file is checked
 * before anything reaches a kernel: format and version, sizes, every
 * transition, failure link, prefix entry and output id inside its machine;
 * a loaded automaton scans exactly as the saved one, with the default scan
 * configuration. Errors: AC_EINVAL (NULL, not such a file, truncated,
 * inconsistent), AC_ERANGE (placement SMEM and a table that does not fit the
 * device), AC_ENOMEM, AC_ECUDA. */
AC_API int ac_load(const char *path, int device, ac_automaton **out);

AC_API int ac_stats(const ac_automaton *a, ac_stats_t *out);

/* Host view of subset k (0 <= k < K). */
AC_API int ac_subset(const ac_automaton *a, uint32_t k, ac_subset_view *out);

/* Set or read the scan configuration used by later scans of `a`. */
AC_API int ac_set_scan_config(ac_automaton *a, const ac_scan_config *cfg);
AC_API int ac_get_scan_config(const ac_automaton *a, ac_scan_config *cfg);

/* Autotune: time candidate configurations on a text of n symbols (device
 * pointer d_text, format fmt) on `stream`, keep the fastest in `a` and
 * return it in *chosen (may be NULL). */
AC_API int ac_tune(ac_automaton *a, const uint8_t *d_text, uint64_t n, int fmt, void *stream,
            ac_scan_config *chosen);

/* ------------------------------------------------------------ scans */

/* Scan n symbols of `text` (fmt AC_U8 or AC_PACKED2; mem AC_HOST or
 * AC_DEVICE) and return the sorted matches and the counts in *out (host
 * arrays, release with ac_result_free). Synchronous: returns when the result
 * is on the host. Host text is copied to the device inside the call; a host
 * text of 32 MiB or more (folded machine) is copied in pieces on a stream of
 * the library's own, and each piece is scanned on `stream` as soon as it has
 * landed (short rows, so that each piece spreads over the GPU), which hides
 * the scan behind the host-to-device copy. Page-locked host memory lets the
 * copies run asynchronously. */
AC_API int ac_scan(const ac_automaton *a, const uint8_t *text, uint64_t n, int fmt, int mem,
            void *stream, ac_result *out);

/* Asynchronous scan, device in and device out, no host synchronisation:
 * queues the work on `stream` and returns. d_matches has room for `cap`
 * records; *d_num_matches (device, uint64) receives the true number of
 * matches M; when M > cap the records are unspecified (retry with cap >= M).
 * *d_num_matches == UINT64_MAX means a device-side wait ran out (error).
 * d_counts (device, num_patterns uint64) may be NULL. Scratch memory comes
 * from the library's stream-ordered pool. */
AC_API int ac_scan_async(const ac_automaton *a, const uint8_t *d_text, uint64_t n, int fmt, void *stream,
                  ac_match *d_matches, uint64_t cap, uint64_t *d_num_matches, uint64_t *d_counts);

/* The two stages of ac_scan_async, for callers that time or overlap them.
 * ac_scan_keys_async: steps of the scan up to the unsorted matches — every
 * match as one uint64 key (pos << ac_key_shift(a)) | pattern_id in d_keys
 * (room for cap keys; order unspecified), the true count M in *d_num (device
 * uint64; UINT64_MAX if a device-side wait ran out) and, if d_counts is not
 * NULL, the per-pattern counts (device, num_patterns uint64, zeroed by the
 * call). Keys beyond cap are dropped (M still counts them). */
AC_API int ac_scan_keys_async(const ac_automaton *a, const uint8_t *d_text, uint64_t n, int fmt, void *stream,
                              uint64_t *d_keys, uint64_t cap, uint64_t *d_num, uint64_t *d_counts);
/* Bits below the position in a key: ceil(log2(num_patterns)), at least 1. */
AC_API int ac_key_shift(const ac_automaton *a);
/* Sort the first min(*d_num, cap) keys of d_keys (device; cap entries, the
 * entries at and beyond *d_num are overwritten) ascending and write them as
 * ac_match records to d_matches (device, cap records); *d_num_out (device,
 * may alias d_num) receives *d_num. n = the text length the keys came from
 * (bounds the sort's key bits). Scratch comes from the library's pool. */
AC_API int ac_sort_keys_async(const ac_automaton *a, uint64_t n, uint64_t *d_keys, const uint64_t *d_num,
                              uint64_t cap, void *stream, ac_match *d_matches, uint64_t *d_num_out);

/* ac_scan_noalloc: the same scan as ac_scan_async, for callers that must
 * not allocate device memory while scanning (the paper has no counterpart;
 * this is a deployment convenience). Some callers cannot call cudaMalloc or
 * cudaMallocAsync at that point: a process whose device memory was reserved
 * in advance by another allocator, a latency-critical loop that cannot take
 * an allocation's implicit synchronisation or lock, or a host application
 * that forbids the library any allocation. This entry point allocates
 * nothing; its scratch is one fixed array of about 8.1 MiB compiled into the
 * library. A device holds that array from the first ac_scan_noalloc call on
 * it until the process exits: the first call on a device loads this part of
 * the library's device code and reserves the array (through
 * cudaGetSymbolAddress), so make it at initialisation -- a call with n = 0
 * and cap = 0 does it -- before the device's memory is committed elsewhere
 * and before any stream capture. If that first lookup fails (AC_ENOMEM when
 * the device has no room, else AC_ECUDA), nothing is kept and the next call
 * tries again. Limits: cap <= 262,144 match records (larger cap:
 * AC_ERANGE); the text must be 16-byte aligned unless it is at most 65,536
 * bytes (else AC_EINVAL).
 * Every call uses the same array, which keeps the previous call's contents
 * (the call clears what must start at zero): calls that overlap on the GPU,
 * from any stream or thread, race and must be serialised by the caller.
 * Arguments, outputs and errors are otherwise those of ac_scan_async. */
AC_API int ac_scan_noalloc(const ac_automaton *a, const uint8_t *d_text, uint64_t n, int fmt, void *stream,
                           ac_match *d_matches, uint64_t cap, uint64_t *d_num_matches, uint64_t *d_counts);

/* One text of a batch. */
typedef struct {
    uint32_t automaton; /* index into the automata array */
    int32_t fmt;        /* AC_U8 or AC_PACKED2 */
    const uint8_t *text;
    uint64_t n;         /* symbols */
} ac_batch_item;

/* Flags of ac_scan_batch. */
#define AC_BATCH_NO_COUNTS 1u /* leave outs[i].counts NULL (no per-text count arrays) */
#define AC_BATCH_GRAPH 2u     /* keep this batch's plan (layout, device buffers, autotuned row length and
                                 CTA shape) and replay it as one CUDA graph when the same batch -- same
                                 automata, same text pointers, lengths and formats -- is scanned again; the
                                 first such call autotunes. At most two plans are kept; ac_batch_release
                                 drops them. Implies AC_BATCH_ONE_LAUNCH. */
#define AC_BATCH_ONE_LAUNCH 4u /* lay every text of an alphabet class out in one arena and scan them in one
                                  persistent launch. Without it (and without AC_BATCH_GRAPH), byte texts
                                  whose alphabet leaves a byte free are scanned one automaton at a time as
                                  one text: the automaton's texts laid end to end, each behind a byte outside
                                  the alphabet (which sends the walk back to the root), through the single-
                                  text path and its kernel choice; packed texts always take the arena. */

/* Scan ni texts, each against one of na resident automata (all built on the
 * same device): byte texts whose alphabet leaves a byte free, one automaton
 * at a time as one text (see AC_BATCH_ONE_LAUNCH); otherwise in one
 * persistent launch per alphabet class: the texts are laid out in one device
 * arena of whole chain rows, grouped by automaton, and a tile list assigns
 * (automaton subset, rows) pairs to persistent CTAs (Section III's input- and
 * pattern-focused splits applied to many texts at once). mem = AC_HOST or
 * AC_DEVICE for all item texts; texts are copied inside the call. outs[i] receives item i's sorted matches
 * (positions relative to item i's text) and, unless AC_BATCH_NO_COUNTS, its
 * counts (sized by its automaton's pattern count). Synchronous. Errors:
 * AC_EINVAL (NULL, bad automaton index or format, automata on different
 * devices), AC_ERANGE (a text of 2^32 symbols or more, a batch too large for
 * one launch), AC_ENOMEM, AC_ECUDA, AC_ETIMEDOUT. On error every outs[i] is
 * left zeroed. */
AC_API int ac_scan_batch(const ac_automaton *const *as, uint32_t na, const ac_batch_item *items,
                         uint32_t ni, int mem, uint32_t flags, void *stream, ac_result *outs);

/* Drop the plans kept by AC_BATCH_GRAPH (their device and pinned memory). */
AC_API void ac_batch_release(void);

/* Release the arrays of a result (NULL or zeroed is a no-op). */
AC_API void ac_result_free(ac_result *r);

/* Move n results into two flat host arrays and release them (as
 * ac_result_free): matches of outs[i] to matches[moff[i] .. moff[i] +
 * outs[i].num_matches), where moff[0] = 0 and moff[i + 1] = moff[i] +
 * outs[i].num_matches (written by the call, n + 1 entries); with counts not
 * NULL, the counts of outs[i] (num_patterns entries, zeros when outs[i] has
 * none) to counts[coff[i] ..), coff likewise over num_patterns (n + 1
 * entries). The caller sizes matches and counts from the results' fields
 * (sum of num_matches, sum of num_patterns). Host memory only. AC_EINVAL for
 * NULL arguments (nothing is moved or released then). */
AC_API int ac_results_take(ac_result *outs, uint32_t n, ac_match *matches, uint64_t *moff, uint64_t *counts,
                           uint64_t *coff);

/* ------------------------------------------------------------ serving */
typedef struct {
    uint64_t device_mem_budget; /* bytes of device memory the server may hold for texts and results
                                   (0 = 4 GiB) */
    uint32_t max_batch_items;   /* most requests coalesced into one launch (0 = 256) */
    uint32_t max_queue;         /* queued requests before submit refuses with AC_EBUSY (0 = 65536) */
    uint32_t num_streams;       /* launches in flight at once (0 = 2) */
    uint32_t max_wait_us;       /* how long the scheduler lets a partial batch wait for more arrivals
                                   (0 = none) */
    uint64_t pinned_bytes;      /* page-locked host staging the server copies submitted texts into when
                                   they are not staged on the device (0 = 1 GiB); texts that fit neither
                                   wait in ordinary host memory */
    uint32_t staging;           /* AC_STAGE_DEVICE (0) or AC_STAGE_PINNED: where ac_serve_submit puts the
                                   text until its batch runs */
} ac_serve_opts;

#define AC_STAGE_DEVICE 0 /* submit copies the text straight into device memory (one host->device copy on
                             the calling thread's per-thread stream, finished before submit returns); at
                             most device_mem_budget bytes of texts wait there, the rest go to the pinned
                             slab */
#define AC_STAGE_PINNED 1 /* submit copies the text into the page-locked slab; the batch's launch copies
                             it to the device */

/* Start a server over na resident automata (borrowed; they must outlive the
 * server). A scheduler thread admits requests by memory, coalesces them into
 * batched launches and completes them. */
AC_API int ac_serve_create(const ac_automaton *const *as, uint32_t na, const ac_serve_opts *opts,
                    ac_server **out);

/* Queue a request: scan host text[0..n) (copied before returning, into
 * device memory or the pinned slab as opts.staging says) with automaton
 * `automaton`. *ticket identifies it. AC_EBUSY when the queue is full,
 * AC_ERANGE when the text alone exceeds the memory budget. */
AC_API int ac_serve_submit(ac_server *s, uint32_t automaton, const uint8_t *text, uint64_t n, int fmt,
                    uint64_t *ticket);

/* ac_serve_submit for a request that arrived before the call: arrival_ns is
 * its arrival time on the host's monotonic clock (CLOCK_MONOTONIC, in ns;
 * e.g. the moment a load generator scheduled it), and the server's latency
 * statistics count from that time instead of from the call, so that time a
 * request spent before reaching the server is not lost. Otherwise as
 * ac_serve_submit. */
AC_API int ac_serve_submit_at(ac_server *s, uint32_t automaton, const uint8_t *text, uint64_t n, int fmt,
                              uint64_t arrival_ns, uint64_t *ticket);

/* Non-blocking: AC_EAGAIN while pending; AC_OK moves the result into *out
 * (the ticket is then consumed). */
AC_API int ac_serve_poll(ac_server *s, uint64_t ticket, ac_result *out);

/* Blocking with a timeout in milliseconds: AC_ETIMEDOUT if not done in time. */
AC_API int ac_serve_wait(ac_server *s, uint64_t ticket, uint32_t timeout_ms, ac_result *out);

/* Counters of a server; p50_ms / p99_ms: latency percentiles of the
 * completed requests, from arrival (the submit call, or the time given to
 * ac_serve_submit_at) to the result on the host. */
typedef struct {
    uint64_t submitted, completed, launches, items_launched, queued, in_flight;
    double p50_ms, p99_ms, mean_batch_items;
} ac_serve_stats_t;

AC_API int ac_serve_stats(ac_server *s, ac_serve_stats_t *out);

/* Stop the scheduler (pending requests complete first) and release everything. */
AC_API void ac_serve_destroy(ac_server *s);

/* ------------------------------------------------------------ roofline probe */

/* The lookup ceilings the scan meets (Section II.A: one dependent goto-table
 * lookup per text symbol; the paper measures CPU throughput only, so this
 * probe has no counterpart there). */
typedef struct {
    double ms;             /* device time of the timed launch (CUDA events) */
    double gathers;        /* dependent 4-byte reads in it: sms * chains_per_sm * steps */
    double gathers_per_s;
    uint32_t chains_per_sm;
    uint32_t sms;
} ac_gather_probe;

/* Measure dependent random 4-byte reads on device `device`: a table of
 * table_bytes (seeded pseudo-random words, allocated and freed by the call)
 * in global memory (shared = 0: served by L2 when the table fits there, else
 * by HBM) or copied into each CTA's shared memory (shared = 1; the table must
 * fit one CTA's shared memory, else AC_ERANGE). One CTA of `threads` threads
 * per SM, each thread walking `chains` (1, 2, 4 or 8) independent chains of
 * `steps` lookups, each lookup's address taken from the word the previous
 * one read. One untimed warm-up launch precedes the timed one. Synchronous.
 * Errors: AC_EINVAL (NULL out, threads not a multiple of 32 in [32, 1024],
 * chains), AC_ERANGE, AC_ENOMEM, AC_ECUDA. */
AC_API int ac_probe_gather(int device, uint64_t table_bytes, int shared, uint32_t threads, uint32_t chains,
                           uint32_t steps, ac_gather_probe *out);

/* The launch floor a chain of scan launches meets: enqueue `launches` empty
 * kernels of `blocks` CTAs x `threads` threads, one after the other, on
 * `stream` (a cudaStream_t; NULL is the legacy default stream) of the
 * current device. Asynchronous; may be captured in a CUDA graph, where each
 * launch is one kernel node depending on the one before it. Replaying a
 * graph of empty nodes shaped like a scan call's device operations gives the
 * time a call spends on launches alone. Errors: AC_EINVAL (launches,
 * blocks or threads 0, threads over 1024), AC_ECUDA (a launch failed). */
AC_API int ac_probe_launch(void *stream, uint32_t launches, uint32_t blocks, uint32_t threads);

/* ------------------------------------------------------------ misc */
AC_API const char *ac_strerror(int code);
AC_API const char *ac_last_error(void);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
AC_API int ac_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AC_H */
