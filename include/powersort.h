/*
 * powersort.h -- C ABI of the GB300 (sm_103a) Powersort library.
 *
 * The library sorts unsigned 32-bit keys stably on the GPU by the method of
 * "Virtual-Memory Powersort" (Moltmann, Nakajima, Wild):
 *   - runs are maximal non-decreasing segments, short ones extended to the
 *     minimum run length and insertion-sorted (Sec. 2 operation ExtractRun;
 *     Sec. 5 "Algorithm variants" for the minrun rule);
 *   - every boundary between adjacent runs gets its Power (Sec. 2 Theorem);
 *   - the runs are merged along the tree that Algorithm 1's stack policy
 *     builds (merge the stack top while its power is >= the new power), with
 *     stable merges that take the left run on ties (Algorithm 2);
 *   - run storage is either Pingpong (Sec. 3: one n-element scratch buffer,
 *     every merge out of place) or virtual-memory pages (Sec. 4: runs as page
 *     lists over a small recycled page pool, a final page permutation).
 * The result is the unique stable sort: sorted keys and, optionally, the
 * stable permutation perm (perm[r] = input index of the r-th output).
 *
 * Conventions for every call below:
 *   - Pointers named d_* are CUDA device pointers owned by the caller; the
 *     library reads and writes them only inside the call's stream work.
 *     Pointers named h_* (and the stats / config structs) are host memory.
 *   - Keys are uint32_t, sorted in place (the paper's Powersort(input[0, n))
 *     sorts its input in place, Algorithm 1).  perm is output only.
 *   - All work is enqueued on the stream given to ps_create.  A call returns
 *     once its work is enqueued, except when it is given a non-NULL stats
 *     pointer or it is a ps_get_* call: those synchronise the stream.
 *   - Errors: a call that returns anything but PS_OK has enqueued nothing
 *     (argument errors) or has left the outputs unspecified (device errors).
 *     PS_EINVAL: NULL where a pointer is required, sizes above the limits
 *     given at create time, offsets not non-decreasing.  PS_ENOMEM: device
 *     allocation failed.  PS_ECUDA: a CUDA call failed.  PS_ETIMEOUT: a
 *     device-side wait exceeded its iteration limit (the kernel stopped and
 *     reported it; the context stays usable).  PS_EINTERNAL: a device-side
 *     consistency check failed.
 *   - Nothing falls back to the CPU: without a usable GPU every call that
 *     needs one returns PS_ECUDA.
 *   - A context is used by one host thread at a time.
 */
#ifndef POWERSORT_H
#define POWERSORT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PS_API __attribute__((visibility("default")))

typedef enum ps_status {
    PS_OK = 0,
    PS_EINVAL = 1,
    PS_ENOMEM = 2,
    PS_ECUDA = 3,
    PS_ETIMEOUT = 4,
    PS_EINTERNAL = 5,
    PS_ECANCELED = 6    /* a server request cancelled before it ran             */
} ps_status;

/* Run storage (Sec. 1 "Pingpong Powersort" and "Virtual-Memory Powersort"). */
typedef enum ps_mode {
    PS_MODE_PINGPONG = 0, /* Sec. 3: scratch of n keys (+ n perm entries)          */
    PS_MODE_VM = 1        /* Sec. 4: page pool of O(sqrt(n log n)) elements + tables */
} ps_mode;

/* How the 32-bit keys are ordered (the key-value generalisation: the keys
 * are sorted as these values; their bit patterns travel unchanged). */
typedef enum ps_key_type {
    PS_KEY_U32 = 0, /* unsigned integers (the default)                            */
    PS_KEY_I32 = 1, /* two's-complement signed integers                           */
    PS_KEY_F32 = 2  /* IEEE 754 binary32 under totalOrder (IEEE 754-2008 Sec. 5.10):
                       -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN; NaNs of one
                       sign ordered by their bit patterns                         */
} ps_key_type;

typedef struct ps_config {
    uint32_t mode;       /* ps_mode                                                  */
    uint32_t want_perm;  /* nonzero: calls may produce the stable permutation        */
    uint64_t max_n;      /* largest instance, >= 1, < 2^32                           */
    uint64_t max_total;  /* largest sum of instance sizes per batched call (0: max_n) */
    uint32_t max_count;  /* most instances per batched call (0: 1)                   */
    uint32_t page_log2;  /* VM page size P = 2^page_log2 (0: chosen from max_n as
                            sqrt(n / log2 n) rounded to a power of two, Sec. 4)      */
    uint32_t tile_log2;  /* on-chip tile capacity 2^tile_log2 in 10..12 (0: 12)      */
    uint32_t pool_pages; /* VM page-pool size in pages (0: chosen by the library; >= 16) */
    uint32_t flags;      /* PS_FLAG_* below                                          */
    uint32_t key_type;   /* ps_key_type of the keys this context sorts               */
    uint32_t merge_lanes; /* HBM merge kernel: most chunks a CTA prepares ahead
                             (its search lanes), 1..16 (0: 16); a tuning knob      */
    uint32_t merge_ctas;  /* HBM merge kernel: CTAs per SM, 1 or 2 (0: 2)          */
} ps_config;

/* ps_config.flags */
#define PS_FLAG_TIMING 1u  /* record CUDA events around every phase (ps_get_phase_times) */
#define PS_FLAG_HOST_IO 2u /* allocate device arrays for ps_run_host (max_total keys + perm) */
/* Run detection also takes strictly decreasing runs and reverses them in
 * place (the variant Sec. 5 "Algorithm variants" names).  A run whose first
 * two elements are strictly decreasing continues while the order stays
 * strictly decreasing; equal neighbours end it, so the sort stays stable.
 * The result is the same stable sort; the runs, powers and merge tree are
 * those of the variant. */
#define PS_FLAG_DESCENDING_RUNS 4u
/* Allocate the arrays ps_sort_records and ps_sort_keys64 need (about 25
 * bytes per element of max_n: window keys, descent mask, group list, merge
 * scratch, the sorted 64-bit rows). */
#define PS_FLAG_RECORDS 8u
#define PS_RECORD_MAX_WORDS 1024u
/* VM storage: the final Copy (Sec. 4) in batches of consecutive target pages
 * -- each target's content first moved out to a free page, then every target
 * filled, the paper's page-by-page order done a batch at a time -- instead of
 * the default walk along the chains of the page permutation (one move per
 * page).  The result is the same; the default is faster, and falls back to
 * this order by itself when the chains do not split into short segments. */
#define PS_FLAG_VM_BATCHED_COPY 16u

/* Per-call statistics (sums over instances for batched calls).  The paper's
 * merge cost M is the sum of the lengths of all merge inputs (Sec. 2
 * Definition); the theorem bounds it by n(H + 2). */
typedef struct ps_stats {
    uint64_t n;             /* elements sorted                                    */
    uint64_t runs;          /* runs found by run detection                        */
    uint64_t merge_cost;    /* M                                                  */
    uint64_t tiles;         /* subtrees merged on chip (one CTA each)             */
    uint64_t global_nodes;  /* merges done through HBM                            */
    uint64_t leaf_moves;    /* elements copied to reach the parity buffer         */
    uint64_t scratch_bytes; /* device memory owned by the context                 */
    uint64_t peak_pages;    /* VM mode: most pool pages in use at once (else 0)   */
    uint32_t max_power;     /* largest boundary power                             */
    uint32_t rounds;        /* HBM merge rounds executed                          */
    uint32_t minrun;        /* minrun of the (first) instance                     */
    uint32_t instances;
    uint64_t hbm_merge_elems; /* sum of the sizes of the merges done through HBM  */
    uint32_t launches;      /* kernels the call launched                          */
    uint32_t pages_spliced; /* VM mode: output pages that took over a whole input
                               page through the page table, moving no element */
    uint32_t page_size;     /* VM mode: P, elements per page (else 0)             */
    uint32_t pool_pages;    /* VM mode: pages of the pre-allocated pool (else 0)  */
    uint64_t copy_pages;    /* VM mode: page moves made by the final Copy (Sec. 4)  */
} ps_stats;

typedef struct ps_ctx ps_ctx;

/* Human-readable name of a status code (static storage). */
PS_API const char* ps_status_str(ps_status s);

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Allocates every
 * device buffer the limits in *cfg can need (Sec. 4 "Pre-allocation of
 * buffers": all extra memory is taken once, up front).  *out receives the
 * context; on error it is set to NULL. */
PS_API ps_status ps_create(const ps_config* cfg, int device, void* cuda_stream, ps_ctx** out);

/* Powersort(input[0, n)) (Algorithm 1): sort d_keys[0, n) in place, stably.
 * d_perm: NULL, or n entries receiving the stable permutation (requires
 * want_perm at create time).  n == 0 and n == 1 are valid.  stats: NULL, or
 * filled after the stream is synchronised. */
PS_API ps_status ps_run(ps_ctx* ctx, uint32_t* d_keys, uint32_t* d_perm, uint64_t n,
                        ps_stats* stats);

/* The same sort for `count` independent instances in one set of launches.
 * Instance q is d_keys[off[q], off[q+1]) where off = d_offsets (device,
 * count + 1 entries, non-decreasing, off[0] = 0); perm values are local to
 * each instance.  count must be <= max_count; the table itself is checked on
 * the device (each size <= max_n, off[count] <= max_total): a bad table makes
 * the call sort nothing, and the next synchronising call (stats, ps_sync)
 * returns PS_EINVAL.  The call never synchronises unless stats is given, so
 * it can be captured into a CUDA graph (see ps_graph_create_batched). */
PS_API ps_status ps_run_batched(ps_ctx* ctx, uint32_t* d_keys, uint32_t* d_perm,
                                const uint64_t* d_offsets, uint32_t count, ps_stats* stats);

/* Payloads of any width follow the keys through the stable permutation:
 * d_dst row r = d_src row perm[r], rows of row_bytes bytes (>= 1).  With
 * d_offsets NULL there is one instance of n rows; otherwise `count`
 * instances laid out as in ps_run_batched (n is ignored; perm values are
 * local to each instance, rows of instance q start at row off[q] of both
 * arrays).  d_src and d_dst must not overlap.  Asynchronous on the
 * context's stream; a permutation entry outside its instance (or a bad
 * offsets table) copies nothing for that row and makes the next
 * synchronising call return PS_EINVAL. */
PS_API ps_status ps_gather_rows(ps_ctx* ctx, const uint32_t* d_perm, const uint64_t* d_offsets, uint32_t count,
                                uint64_t n, const void* d_src, void* d_dst, uint32_t row_bytes);

/* Records: rows of `words` 32-bit words (row i = d_rec[i * words, (i + 1) *
 * words)), ordered lexicographically with the words as unsigned integers
 * (the paper's blob types, Sec. 5 "Input data types").  d_perm receives the
 * stable order (n entries); d_rec_out, if not NULL, the rows in that order
 * (n * words words; it must not overlap d_rec, which is read only).  The runs,
 * powers, merge tree and merge cost (ps_get_*) are those of Algorithm 1 on
 * the records; the rows move once, at the end.  Needs a context made with
 * PS_FLAG_RECORDS and want_perm, keys of type PS_KEY_U32 and no
 * PS_FLAG_DESCENDING_RUNS; 1 <= words <= PS_RECORD_MAX_WORDS, n <= max_n.
 * Asynchronous unless stats is given. */
PS_API ps_status ps_sort_records(ps_ctx* ctx, const uint32_t* d_rec, uint32_t words, uint64_t n,
                                 uint32_t* d_perm, uint32_t* d_rec_out, ps_stats* stats);

/* 64-bit keys: sort d_keys[0, n) in place, stably, read as key_type's
 * 64-bit counterpart (PS_KEY_U32: unsigned, PS_KEY_I32: two's complement,
 * PS_KEY_F32: IEEE 754 binary64 under totalOrder); d_perm receives the
 * stable permutation.  A 64-bit key is a record of two words (high, low),
 * so this runs the record sort on an order-preserving image of the keys:
 * runs, powers, merge tree and merge cost are Algorithm 1's on the 64-bit
 * keys.  Needs a context made with PS_FLAG_RECORDS and want_perm (and the
 * context's own key_type PS_KEY_U32).  Asynchronous unless stats is given. */
PS_API ps_status ps_sort_keys64(ps_ctx* ctx, uint64_t* d_keys, uint64_t n, uint32_t* d_perm, uint32_t key_type,
                                ps_stats* stats);

/* A batched sort captured once into a CUDA graph and replayed with one
 * launch (its arrays are fixed at capture time; refill them between
 * launches).  ps_graph_create_batched captures ps_run_batched(ctx, d_keys,
 * d_perm, d_offsets, count) on the context's stream (which must not be
 * capturing already) and instantiates it; ps_graph_launch enqueues one
 * replay on the context's stream (asynchronous: use ps_sync, or stats
 * through ps_get_instance_stats); ps_graph_destroy frees it (NULL: no-op).
 * Phase timing (PS_FLAG_TIMING) is not recorded inside a graph. */
typedef struct ps_graph ps_graph;
PS_API ps_status ps_graph_create_batched(ps_ctx* ctx, uint32_t* d_keys, uint32_t* d_perm,
                                         const uint64_t* d_offsets, uint32_t count, ps_graph** out);
PS_API ps_status ps_graph_launch(ps_graph* g);
PS_API void ps_graph_destroy(ps_graph* g);

/* ps_run for host arrays: copies h_keys[0, n) to the device, sorts, and
 * copies the sorted keys (and, if h_perm is not NULL, the permutation) back;
 * returns after the copies have finished.  Needs PS_FLAG_HOST_IO at create
 * time.  Pinned (page-locked) host memory gives full-speed copies. */
PS_API ps_status ps_run_host(ps_ctx* ctx, uint32_t* h_keys, uint32_t* h_perm, uint64_t n, ps_stats* stats);

/* Durations in milliseconds of the phases of the last call (needs
 * PS_FLAG_TIMING; synchronises): [0] setup, [1] run detection, [2] powers and
 * merge schedule, [3] on-chip tiles, [4] HBM merge rounds, [5] statistics.
 * Measured with CUDA events recorded on the context's stream between the
 * launches.  h_ms receives min(cap, 6) values; *count (may be NULL) gets 6. */
PS_API ps_status ps_get_phase_times(ps_ctx* ctx, float* h_ms, uint32_t cap, uint32_t* count);

/* Timeline of the HBM merges of the last call (synchronises), four values
 * per round that ran, in microseconds since the merge kernel started.
 * Pingpong: the merges are grouped in rounds of equal power (children before
 * parents) but run as a dataflow: a merge starts when its two children are
 * complete, so rounds overlap; the values are the first and the last time
 * one of the round's chunks found its inputs complete, and the first and the
 * last time one of its chunks sent its output.  VM storage: the rounds are
 * separated by grid barriers; the values are the round's start, the start of
 * its page dataflow (after the page marks, records, splits and the list of
 * touched pages), the end of the page dataflow, and the round's end.  h_us
 * receives min(cap, 4 x rounds) values; *count (may be NULL) gets 4 x rounds. */
PS_API ps_status ps_get_round_times(ps_ctx* ctx, float* h_us, uint32_t cap, uint32_t* count);

/* Wait for the context's stream and report the device-side status of the
 * last call: PS_OK, or PS_ETIMEOUT / PS_EINTERNAL when a kernel gave up a
 * bounded wait or failed a consistency check (calls without stats return
 * after enqueueing, so this is where such errors surface). */
PS_API ps_status ps_sync(ps_ctx* ctx);

/* Failure detection, exercised on purpose: a cooperative launch of two CTAs
 * in which one never arrives at the grid barrier the other waits at (the
 * same barrier and spin limit every persistent kernel of the library uses).
 * The waiting CTA gives up after the limit (about two seconds), records the
 * timeout and returns; the call returns PS_ETIMEOUT and the context stays
 * usable (the next sort resets the device status).  No GPU fault, trap or
 * hang is involved. */
PS_API ps_status ps_selftest_wait_timeout(ps_ctx* ctx);

/* Canary words after every device buffer the context owns (with
 * PS_FLAG_RECORDS, also those of the inner context of its nested sort):
 * PS_OK while they hold their pattern, PS_EINTERNAL if a kernel wrote past a
 * buffer's end (synchronises). */
PS_API ps_status ps_check_guards(ps_ctx* ctx);

/* Introspection of the last call, for parity checks (synchronises).
 *   ps_get_runs:   run starts of instance q plus its end (runs + 1 entries),
 *                  instance-local (ExtractRun, Sec. 2 / Sec. 5).
 *   ps_get_powers: Power of every boundary between adjacent runs of instance
 *                  q, left to right (runs - 1 entries, Sec. 2 Theorem).
 *   ps_get_nodes:  for every boundary, the element range [lo, hi) of the
 *                  merge that joins its two sides in Algorithm 1 (2 entries
 *                  per boundary: lo, hi), i.e. the merge tree.  The sort keeps
 *                  only its HBM merges, so this call recomputes every range on
 *                  the device with the planning's own code, in a temporary
 *                  device buffer of 8 bytes per boundary (PS_ENOMEM if it
 *                  cannot be had).
 * h_out receives at most `cap` entries; *count (may be NULL) receives the
 * number available.  PS_EINVAL if q is not an instance of the last call. */
PS_API ps_status ps_get_runs(ps_ctx* ctx, uint32_t q, uint32_t* h_out, uint64_t cap,
                             uint64_t* count);
PS_API ps_status ps_get_powers(ps_ctx* ctx, uint32_t q, uint8_t* h_out, uint64_t cap,
                               uint64_t* count);
PS_API ps_status ps_get_nodes(ps_ctx* ctx, uint32_t q, uint32_t* h_out, uint64_t cap,
                              uint64_t* count);
/* Statistics of one instance of the last call (synchronises). */
PS_API ps_status ps_get_instance_stats(ps_ctx* ctx, uint32_t q, ps_stats* stats);

/* Device memory the context owns, in bytes: every buffer ps_create allocated
 * (the figure ps_stats.scratch_bytes reports after a call).  No kernel runs
 * and nothing synchronises, so it can be asked right after ps_create (the
 * server charges its lanes with it against the budget). */
PS_API ps_status ps_get_scratch_bytes(const ps_ctx* ctx, uint64_t* bytes);

/* Release every device buffer of the context.  NULL is a no-op. */
PS_API void ps_destroy(ps_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Serving: independent sorts of host arrays, continuously batched.  The
 * server keeps `lanes` batched contexts (each with its own stream and device
 * arrays, sized so that all lanes together stay within budget_bytes of device
 * memory).  A dispatcher thread fills every idle lane with queued requests in
 * arrival order (as many as fit lane_max_total elements and lane_max_count
 * requests) and enqueues their host->device copies, one batched sort and the
 * device->host copies of the results; lanes run concurrently, so requests
 * arriving while others are on the GPU are admitted as lanes free up.
 * Results are the same stable sort that ps_run computes.  The memory charged
 * against budget_bytes is what the lanes really hold: each lane's input and
 * output arrays and offsets table plus its context's ps_get_scratch_bytes. */
typedef struct ps_server ps_server;
typedef struct ps_server_config {
    uint64_t budget_bytes;   /* device memory the server may hold                  */
    uint64_t max_n;          /* largest request, < 2^32                            */
    uint64_t lane_max_total; /* elements per batch (0: from the budget, <= 2^28)   */
    uint32_t lane_max_count; /* requests per batch (0: 1024)                       */
    uint32_t lanes;          /* batches in flight at once (0: 4)                   */
    uint32_t want_perm;      /* nonzero: requests may ask for the permutation      */
    uint32_t device;
    uint32_t key_type;       /* ps_key_type of every request's keys                */
    uint32_t flags;          /* PS_FLAG_DESCENDING_RUNS or 0                      */
    uint32_t storage;        /* ps_mode of the lanes' contexts (0: Pingpong).  With
                                PS_MODE_VM a lane holds a page pool and tables
                                instead of Pingpong's n-element scratch (about 8
                                bytes per element), so a budget admits about twice
                                the elements per lane.  A request of more than 2^20
                                elements is then a batch by itself, sorted with paged
                                storage (Sec. 4: one instance per call); smaller
                                ones are batched (at most 2^22 elements) in a small
                                Pingpong context the lane also holds              */
    uint32_t reserved;
} ps_server_config;

typedef struct ps_server_stats {
    uint64_t submitted, completed, failed, elements, batches, queued;
    uint64_t device_bytes;   /* device memory held by the lanes (<= budget_bytes)  */
    uint64_t lane_max_total;
    uint32_t lanes;
    uint32_t max_busy_lanes; /* most lanes seen busy at once (overlap evidence)    */
} ps_server_stats;

/* Cancel a queued request: PS_OK when it had not left the queue (its wait /
 * poll then return PS_ECANCELED and it counts as failed), PS_EINVAL when the
 * ticket is unknown or the request is already on the GPU or done. */
PS_API ps_status ps_server_cancel(ps_server* srv, uint64_t ticket);

/* Start a server (allocates every lane up front; PS_ENOMEM if the lanes do not
 * fit the budget).  Tracing: when the environment variable PS_SERVER_TRACE
 * names a file, the server records every batch (lane, requests, elements, the
 * host times it was enqueued and seen complete, and device event times of its
 * first copy in, copies in done, sort start, sort end and copies out done)
 * and writes them there as CSV when it is destroyed. */
PS_API ps_status ps_server_create(const ps_server_config* cfg, ps_server** out);
/* Queue one sort: h_in[0, n) is read (not modified); the sorted keys go to
 * h_keys_out and, if h_perm_out is not NULL, the stable permutation to
 * h_perm_out.  All three host arrays must stay valid until the ticket
 * completes; page-locked memory makes the copies asynchronous. */
PS_API ps_status ps_server_submit(ps_server* s, const uint32_t* h_in, uint32_t* h_keys_out, uint32_t* h_perm_out,
                                  uint64_t n, uint64_t* ticket);
/* *done = 1 once the ticket has completed (its outputs are written);
 * *latency_s (may be NULL) = seconds from submission to completion. */
PS_API ps_status ps_server_poll(ps_server* s, uint64_t ticket, int* done, double* latency_s);
/* Block until the ticket completes (PS_ETIMEOUT after timeout_s seconds). */
PS_API ps_status ps_server_wait(ps_server* s, uint64_t ticket, double timeout_s, double* latency_s);
PS_API ps_status ps_server_get_stats(ps_server* s, ps_server_stats* out);
/* Drain the queue, stop the dispatcher and free every lane. */
PS_API void ps_server_destroy(ps_server* s);

/* ---------------------------------------------------------------------------
 * Sorting without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code that
 * owns a fixed, pre-sized budget of device memory which a foreign
 * allocation would overrun, and latency-sensitive loops in which
 * cudaMalloc / cudaFree would synchronise the device.
 *
 * ps_run_noalloc sorts d_keys[0, n) in place, stably, and writes the stable
 * permutation to d_perm (NULL: keys only) -- the same result as ps_run --
 * using one CTA on device `device`, enqueued on `cuda_stream` (a
 * cudaStream_t; NULL = legacy default stream).  It needs no context and
 * allocates nothing: its scratch is a file-scope static device array of
 * about 2 MiB that every GPU loading the library holds until the process
 * exits.  n must be <= PS_NOALLOC_MAX_N, else PS_EINVAL and nothing is
 * enqueued.  The first call on a device does a one-time set-up (it looks up
 * the scratch array's device address); make that first call before any
 * stream capture.  Every call shares the one scratch array: calls whose work
 * overlaps on the GPU race and must be serialised by the caller.  The call
 * returns once the kernel is enqueued. */
#define PS_NOALLOC_MAX_N 262144u
PS_API ps_status ps_run_noalloc(uint32_t* d_keys, uint32_t* d_perm, uint64_t n, int device,
                                void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* POWERSORT_H */
