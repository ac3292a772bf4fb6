/*
 * domagg.h -- C ABI of the GB300 (sm_103a) library for aggregation over
 * dominated points.
 *
 * The operation (Sroka & Tyszkiewicz, "Aggregating over Dominated Points by
 * Sorting, Scanning, Zip and Flat Maps", Sec. 1.2): given data points D and
 * queries Q in R^m, weights w on D and an associative, commutative F with
 * unit e, compute for every query q
 *
 *     out(q) = F over { w(d) : d in D, d_i < q_i for every i }   (strict).
 *
 * It is computed the way the paper's algorithm does (Sec. 4, with the
 * one-logarithm improvement of Sec. 5): dense ranks of the first m-1
 * coordinates, a flat map of every point to the canonical range-tree nodes of
 * its ranks (P0 sets for data, P1 sets for queries, Sec. 3), a stable radix
 * sort of those records by node and last coordinate (queries before data on
 * a tie), a segmented scan of F over each node, and a per-query reduction of
 * the partial results.  Every step runs in this library's CUDA kernels.
 *
 * Conventions shared by all entry points
 *   - Coordinates are row-major [n][m] arrays (a contiguous torch (n, m)
 *     tensor), int32 or float32.  -0.0 equals +0.0; +-inf are ordered; a NaN
 *     coordinate makes the call fail with DOMAGG_ERR_NAN.
 *   - Pointers marked "device" are CUDA device memory owned by the caller and
 *     must stay valid until the work on `stream` has finished.  The library
 *     never frees caller memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *     entry points enqueue work on it.  domagg_forward and domagg_backward
 *     synchronise the stream once in mid-call (they read the record count to
 *     size their workspace) and return with the rest of the work enqueued;
 *     outputs are valid once the stream has been synchronised.
 *   - Supported (op, weight dtype) -> output dtype:
 *       SUM   int64 -> int64 (wraps modulo 2^64), float32 -> float32
 *       MAX   int32 -> int32, float32 -> float32
 *       MIN   int32 -> int32, float32 -> float32
 *       COUNT (weights ignored, may be NULL) -> int64
 *     The empty set gives e: 0 for SUM and COUNT, INT32_MIN or -inf for MAX,
 *     INT32_MAX or +inf for MIN; a NaN weight never wins a MAX or a MIN.
 *     float32 sums carry a float-float (hi, lo) accumulator through the scan
 *     and the per-query reduction; the result is within 2^-23 * sum |w(d)|
 *     over the dominated set of the exact sum.  float32 weights must be
 *     finite for SUM.
 *   - m is 1 to 4 (m = 1 is ordinary prefix aggregation, Sec. 1.1).  For
 *     m = 4 the node key (b_1 - 1 + b_2 + b_3 bits) must fit 63 bits, so
 *     the first three coordinates may have at most about 2^21 distinct
 *     values each (DOMAGG_ERR_UNSUPPORTED otherwise).
 *     nD + nQ must be below 2^31 per problem, and the number of flat-map
 *     records below 2^32 per call (DOMAGG_ERR_UNSUPPORTED otherwise).
 *   - Errors are returned, never raised or aborted on.  Errors found on the
 *     device after the mid-call synchronisation (a bounded wait that ran out)
 *     are reported by the next call on the handle or by domagg_sync_status.
 *   - A handle may be used by one host thread at a time.  Calls on one handle
 *     share its workspace, so work from two calls must not overlap on the
 *     device (use one stream per handle, or one handle per stream).
 */
#ifndef DOMAGG_H
#define DOMAGG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DOMAGG_OK = 0,
    DOMAGG_ERR_INVALID_ARG = 1, /* bad pointer, size, dtype, op or m */
    DOMAGG_ERR_UNSUPPORTED = 2, /* m > 4, more than 2^31 points, 2^32 records */
    DOMAGG_ERR_OOM = 3,         /* workspace could not be allocated / over the cap */
    DOMAGG_ERR_CUDA = 4,        /* a CUDA runtime call failed (see domagg_last_error) */
    DOMAGG_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
    DOMAGG_ERR_NAN = 6,         /* a coordinate is NaN */
    DOMAGG_ERR_BOUNDS = 7       /* checked build only: a kernel met an index outside its buffer
                                   (the access was skipped; outputs are undefined) */
} domagg_status;

typedef enum { DOMAGG_SUM = 0, DOMAGG_MAX = 1, DOMAGG_COUNT = 2, DOMAGG_MIN = 3 } domagg_op;

typedef enum { DOMAGG_I32 = 0, DOMAGG_I64 = 1, DOMAGG_F32 = 2 } domagg_dtype;

typedef struct domagg_ctx* domagg_handle;

/* Creates a handle bound to CUDA device `device`.  The handle owns a device
 * workspace, grown on demand and released by domagg_destroy.
 * max_workspace_bytes caps that workspace (0 = no cap); a call that would
 * need more returns DOMAGG_ERR_OOM.  *out receives the handle. */
domagg_status domagg_create(domagg_handle* out, int device, size_t max_workspace_bytes);

/* Frees the workspace and the handle (waits for the handle's work first). */
domagg_status domagg_destroy(domagg_handle h);

/* Aggregation over dominated points (Sec. 1.2) for one problem.
 *   d_coords  device [nD][m] (coord_dtype)   data points D
 *   q_coords  device [nQ][m] (coord_dtype)   queries Q
 *   d_weights device [nD] (weight_dtype)     w(d); ignored for COUNT
 *   out       device [nQ] (output dtype above), overwritten
 * nD or nQ may be 0.  The algorithm: Sec. 4 instructions 0 .. 6m+5 with the
 * Sec. 5 change (last coordinate kept as a value; queries first on ties). */
domagg_status domagg_forward(domagg_handle h, int m, const void* d_coords, int64_t nD,
                             const void* q_coords, int64_t nQ, domagg_dtype coord_dtype,
                             const void* d_weights, domagg_dtype weight_dtype, domagg_op op,
                             void* out, void* stream);

/* domagg_forward with a choice of comparison per coordinate and of variant.
 *   nonstrict_mask  bit i set: coordinate i is compared as d_i <= q_i instead
 *                   of d_i < q_i (bits >= m must be 0).  The paper defines
 *                   the strict order only; a non-strict coordinate among the
 *                   first m-1 gets ranks 2r (data) and 2r+1 (queries), one
 *                   more rank digit, and a non-strict last coordinate puts
 *                   data before queries on ties (the Sec. 4 order).
 *   variant         DOMAGG_IMPROVED: the pipeline of domagg_forward (Sec. 5).
 *                   DOMAGG_BASIC: the unimproved algorithm of Sec. 4: every
 *                   one of the m coordinates becomes a bitstring, records are
 *                   keyed by m node ids (n log^m n of them, data before
 *                   queries within a node tuple); m <= 3.  Same results,
 *                   more records: a cross-check of Lemma 2 at scale.
 *                   DOMAGG_WAVELET: m <= 2 only (else DOMAGG_ERR_UNSUPPORTED).
 *                   The levels of the first coordinate's rank (the P0/P1
 *                   decomposition of Sec. 5) are evaluated on the points
 *                   themselves, two levels per pass from the top: the points,
 *                   kept in the order (rank prefix, last coordinate), get one
 *                   segmented scan per level and a stable partition by the
 *                   rank digit between passes.  No flat-map records are
 *                   materialised; every pass moves 16 bytes per point.  Same
 *                   results (the float32 sum within the same bound).
 * Other arguments, layouts and errors as domagg_forward. */
typedef enum { DOMAGG_IMPROVED = 0, DOMAGG_BASIC = 1, DOMAGG_WAVELET = 2 } domagg_variant;
domagg_status domagg_forward_ex(domagg_handle h, int m, const void* d_coords, int64_t nD,
                                const void* q_coords, int64_t nQ, domagg_dtype coord_dtype,
                                const void* d_weights, domagg_dtype weight_dtype, domagg_op op,
                                uint32_t nonstrict_mask, domagg_variant variant, void* out,
                                void* stream);

/* One shard of domagg_forward, for a forward split over several GPUs (the
 * paper's Sec. 6 reading: the flat map is partitioned and one exchange of the
 * outputs joins the parts).  Every shard runs the point phase on all points
 * (ranks, the order of the last coordinate); the flat map's records are
 * split by node: with gS the rank levels taken per group of 2^gS ranks in
 * shared memory (m = 2; 0 otherwise), shard s takes the levels lv >= gS of
 * the first rank with (lv - gS) % nshards == s and the groups g with
 * g % nshards == s (m = 1 has a single level: shard 0 takes it and the
 * others return the unit).  The shard's outputs are F over its records only;
 * F over the nshards outputs (domagg_combine, or a collective with F) is
 * domagg_forward's result.
 *   shard, nshards  0 <= shard < nshards <= 64
 *   out             device [nQ] (output dtype as domagg_forward), overwritten
 *   out_lo          float32 SUM only: device float32 [nQ], the low halves of
 *                   the shard's float-float partials (out holds the high
 *                   halves), so that joining shards adds no rounding; must be
 *                   NULL or is ignored for other ops.
 * Other arguments, layouts and errors as domagg_forward. */
domagg_status domagg_forward_shard(domagg_handle h, int shard, int nshards, int m, const void* d_coords, int64_t nD,
                                   const void* q_coords, int64_t nQ, domagg_dtype coord_dtype, const void* d_weights,
                                   domagg_dtype weight_dtype, domagg_op op, void* out, float* out_lo, void* stream);

/* The two-sample distance of empirical CDFs (Sec. 1.2 names ECDFs as an
 * application of dominance counting): *d_out = max over z < nz of
 * |count_x[z] / nx - count_y[z] / ny|, with count_x, count_y (device int64
 * [nz], e.g. the COUNT outputs of domagg_forward_ex with every coordinate
 * non-strict and queries X u Y) the points of the samples (sizes nx, ny > 0)
 * dominated by each z.  d_out: one device double, overwritten (0 when
 * nz = 0).  Asynchronous on `stream`; DOMAGG_ERR_INVALID_ARG for null
 * pointers or non-positive sample sizes. */
domagg_status domagg_ecdf_distance(domagg_handle h, const int64_t* count_x, const int64_t* count_y, int64_t nz,
                                   int64_t nx, int64_t ny, double* d_out, void* stream);

/* out[q] = F over parts[s][q], s < nparts (1..64): joins the outputs of
 * domagg_forward_shard.  parts and parts_lo are HOST arrays of nparts device
 * pointers; parts_lo (float32 SUM, may be NULL) holds the low halves.  The
 * float32 sum adds the float-float pairs in float-float and rounds once.
 * Asynchronous on `stream`. */
domagg_status domagg_combine(domagg_handle h, domagg_op op, domagg_dtype weight_dtype, int nparts,
                             const void* const* parts, const float* const* parts_lo, int64_t nQ, void* out,
                             void* stream);

/* Same as domagg_forward with HOST buffers (pageable or pinned): copies the
 * inputs to the handle's device staging area, runs the forward on `stream`,
 * copies `out` back and synchronises before returning.  The weights are
 * copied on a stream of the handle beside the point phase (nothing reads
 * them before the count scan); the call reads the host buffers only until
 * it returns. */
domagg_status domagg_forward_host(domagg_handle h, int m, const void* d_coords, int64_t nD,
                                  const void* q_coords, int64_t nQ, domagg_dtype coord_dtype,
                                  const void* d_weights, domagg_dtype weight_dtype, domagg_op op,
                                  void* out, void* stream);

/* Adjoint of the float32 dominance SUM with respect to the weights:
 *     grad_w[d] = sum of grad_out[q] over queries q with d < q (strict),
 * the reverse-dominance aggregation.  It is computed by the same pipeline with
 * the roles of D and Q swapped and every coordinate key negated (bitwise NOT
 * of its order-preserving key), the records being recomputed, not stored.
 *   grad_out device float32 [nQ]; grad_w device float32 [nD], overwritten. */
domagg_status domagg_backward(domagg_handle h, int m, const void* d_coords, int64_t nD,
                              const void* q_coords, int64_t nQ, domagg_dtype coord_dtype,
                              const float* grad_out, float* grad_w, void* stream);

/* domagg_backward with coordinates compared non-strictly (bit i of
 * nonstrict_mask: d_i <= q_i), the adjoint of domagg_forward_ex's SUM with
 * the same mask, computed by `variant`: DOMAGG_IMPROVED (the Sec. 5
 * pipeline) or DOMAGG_WAVELET (the level-wise formulation, m <= 2);
 * DOMAGG_BASIC returns DOMAGG_ERR_UNSUPPORTED. */
domagg_status domagg_backward_ex(domagg_handle h, int m, const void* d_coords, int64_t nD,
                                 const void* q_coords, int64_t nQ, domagg_dtype coord_dtype,
                                 const float* grad_out, float* grad_w, uint32_t nonstrict_mask,
                                 domagg_variant variant, void* stream);

/* One problem of a batch (all pointers device memory, as in domagg_forward). */
typedef struct {
    int m;
    int64_t nD, nQ;
    const void* d_coords;
    const void* q_coords;
    const void* d_weights;
    void* out;
} domagg_instance;

/* k independent problems in one call: every phase of the pipeline runs as one
 * segmented launch over all instances with the same m (instances never mix:
 * sorts, scans and reductions restart at instance boundaries).  `inst` is a
 * host array of k descriptors; coord/weight dtype and op are shared.  Like
 * domagg_forward, the call synchronises `stream` once per group of
 * instances with the same m (to read their record counts) and once more per
 * record chunk when the records of a group do not fit the workspace at once
 * (a chunk holds whole instances); the remaining work is left enqueued. */
domagg_status domagg_batch(domagg_handle h, int k, const domagg_instance* inst,
                           domagg_dtype coord_dtype, domagg_dtype weight_dtype, domagg_op op,
                           void* stream);

/* A planned batch: the same k problems (same descriptors: pointers and sizes)
 * run again and again -- for instance replayed from a CUDA graph -- with the
 * contents of their buffers free to change between runs.  The paper has no
 * counterpart (it is the pipeline of domagg_batch, Sec. 4 with Sec. 5, with
 * its host-side layout step moved to the device).
 *
 * domagg_batch_plan runs the batch on `stream` twice (writing the outputs
 * each time) and returns when both runs have finished: the first run
 * measures every instance's record counts; the plan then reserves, in a
 * private workspace on `device`, room for (1 + headroom) times those counts
 * (plus 1024) per record chunk and key class (m >= 3: node keys of up to 31
 * bits, and wider ones), and the second, planned run allocates that
 * workspace for good.  headroom >= 0.  The descriptors in `inst` are copied;
 * the buffers they point to must outlive the plan.
 *
 * domagg_plan_run enqueues one planned run on `stream`: kernel launches only
 * -- no synchronisation, no allocation, no host<->device copy -- so it can be
 * captured into a CUDA graph and replayed.  The record layout is computed on
 * the device from the current record counts.  If a run meets more records
 * of a key class (or query records) in a chunk than the plan reserved, the kernels of that
 * chunk write nothing outside the workspace, its outputs are undefined, and
 * DOMAGG_ERR_OOM is recorded for domagg_plan_status.  Device errors of a run
 * (NaN coordinates, a bounded wait that ran out, capacity) are only reported
 * by domagg_plan_status.  Runs of one plan must not overlap on the device
 * (one stream, or graph launches ordered on one stream).
 *
 * domagg_plan_status synchronises `stream` and returns (and clears) the first
 * device-side error recorded by the plan's runs, or DOMAGG_OK.
 * domagg_plan_last_error(p) describes the plan's last error; with p = NULL,
 * the last failed domagg_batch_plan of the calling thread.
 * domagg_plan_workspace_bytes returns the device bytes the plan holds.
 * domagg_plan_destroy waits for the device and frees the plan. */
typedef struct domagg_plan_s* domagg_plan;

domagg_status domagg_batch_plan(domagg_plan* out, int device, int k, const domagg_instance* inst,
                                domagg_dtype coord_dtype, domagg_dtype weight_dtype, domagg_op op,
                                double headroom, void* stream);
domagg_status domagg_plan_run(domagg_plan p, void* stream);
/* Picks, per group of instances with the same m, the fastest of nine launch
 * shapes (2, 4 or 8 radix-sort ranges per resident CTA x 8, 16 or 32
 * flat-map / reduction blocks per SM) by timing planned runs on `stream`
 * (each shape: one warm-up and two timed runs, writing the outputs); later
 * runs use it.  Synchronises; not capturable.  *best_ms (may be NULL)
 * receives the summed time of the chosen shapes. */
domagg_status domagg_plan_autotune(domagg_plan p, void* stream, double* best_ms);
domagg_status domagg_plan_status(domagg_plan p, void* stream);
const char* domagg_plan_last_error(domagg_plan p);
int64_t domagg_plan_workspace_bytes(domagg_plan p);
domagg_status domagg_plan_destroy(domagg_plan p);

/* Self-test of the device-side wait limits (the paper has no counterpart):
 * runs one thread that waits on something that never happens -- which = 0:
 * a decoupled look-back on a predecessor status nothing publishes; which =
 * 1: an mbarrier phase whose bytes are never sent -- and returns what
 * domagg_sync_status then reports: DOMAGG_ERR_TIMEOUT when the wait gave up
 * as designed (after about a second), with the handle still usable.
 * Synchronises `stream`. */
domagg_status domagg_selftest_timeout(domagg_handle h, int which, void* stream);

/* Synchronises `stream` and returns the first device-side error recorded by
 * this handle's kernels since the last check (DOMAGG_ERR_TIMEOUT,
 * DOMAGG_ERR_NAN), or DOMAGG_OK; clears it. */
domagg_status domagg_sync_status(domagg_handle h, void* stream);

/* Human-readable description of the last error on the handle ("" if none).
 * The string is owned by the handle and valid until its next call. */
const char* domagg_last_error(domagg_handle h);

/* Facts about the last forward/backward call, for tests and benchmarks. */
typedef struct {
    int64_t n_points;      /* nD + nQ */
    int64_t n_records;     /* T: records of the flat map */
    int64_t n_query_records; /* records that came from queries */
    int32_t m;
    int32_t rank_bits[3];  /* b_i = ceil(log2 U_i) for the first m-1 dimensions */
    int64_t distinct[3];   /* U_i */
    int32_t record_key_bits; /* bits of the node key sorted by the record sort */
    int32_t record_passes;   /* radix passes over the records */
    int64_t workspace_bytes; /* device workspace currently held by the handle */
    int64_t n_records_shared; /* m = 2, 3: records formed, sorted and scanned in shared memory
                                 (the groups' and the top-level tiles'); the rest of n_records go
                                 through HBM (for a shard: also those left to the other shards) */
} domagg_stats;

domagg_status domagg_get_stats(domagg_handle h, domagg_stats* out);

/* Kernel timing.  When enabled, every launch is bracketed by CUDA events on
 * the launching stream and grouped by kernel kind.  domagg_timing_read
 * synchronises, then returns per kind the number of launches, the summed
 * device time (ms) and the summed algorithmic bytes (the bytes each launch
 * must read and write at minimum), and resets the counters.  Kinds are
 * indexed as in domagg_timing_kind_name. */
#define DOMAGG_TIMING_KINDS 20
typedef struct {
    int32_t launches[DOMAGG_TIMING_KINDS];
    double ms[DOMAGG_TIMING_KINDS];
    double bytes[DOMAGG_TIMING_KINDS];
} domagg_timing;

domagg_status domagg_timing_enable(domagg_handle h, int enable);
domagg_status domagg_timing_read(domagg_handle h, domagg_timing* out);
const char* domagg_timing_kind_name(int kind);

/* Forward pass that allocates nothing: no cudaMalloc, cudaFree, pinned host
 * memory or allocating library routine.  It is for callers that cannot
 * allocate device memory (an allocator-free runtime, a process that reserves
 * all device memory up front, a latency-critical path that must not block in
 * the allocator).  The paper has no counterpart: it is the same pipeline as
 * domagg_forward, with every buffer taken from one file-scope device array of
 * 32 MiB that each GPU loading this library holds until the process exits.
 *   Arguments, layouts, outputs and tolerances are those of domagg_forward;
 *   all pointers are device memory on the CURRENT device, and no handle is
 *   used.
 *   Limits: nD + nQ <= 65536 (checked before any GPU work), and the flat
 *   map must fit the scratch (about 10^6 records for m <= 2, about half that
 *   for m = 3).  The flat map's size is only known once the point phase has
 *   run on the GPU and the mid-call synchronisation has read the record
 *   counts: an input whose records do not fit then returns
 *   DOMAGG_ERR_UNSUPPORTED without writing `out`, and the next call is
 *   unaffected.  Errors are reported by the status code only (there is no
 *   handle to ask domagg_last_error).
 *   The first call on a device sets that device's scratch up (looks its
 *   address up, clears the control block and the status words, and
 *   synchronises the device): make that first call before any CUDA-graph
 *   stream capture.
 *   Every call shares the one array and it keeps the last call's contents;
 *   calls that overlap on the GPU (on different streams, or from several
 *   host threads whose work is not ordered) race and corrupt each other's
 *   results.  Host calls are serialised by a lock; order their GPU work on
 *   one stream.  The call synchronises `stream` once in mid-call, like
 *   domagg_forward. */
domagg_status domagg_forward_noalloc(int m, const void* d_coords, int64_t nD, const void* q_coords, int64_t nQ,
                                     domagg_dtype coord_dtype, const void* d_weights, domagg_dtype weight_dtype,
                                     domagg_op op, void* out, void* stream);

/* Tuning knobs of a handle (the paper has no counterpart); every setting
 * computes the same results:
 *   "group_bits"     0 .. 13 (default 13): for m = 2 and m = 3, the first
 *                    rank's levels below gS <= group_bits (nodes of at most
 *                    2^gS ranks) are formed, sorted and scanned per group of
 *                    2^gS ranks in shared memory (a group too large for it,
 *                    from heavy ties, sends its points' records of those
 *                    levels through HBM); 0 sends every level's records
 *                    through HBM;
 *   "top_bits"       0 .. 12 (default 12): for m = 2, the rank levels from
 *                    tS = max(gS, b0 - top_bits) up are formed, sorted and
 *                    scanned per tile of points in the order of the last
 *                    coordinate in shared memory, with each node's running
 *                    F carried across tiles and ranges of tiles; 0 sends
 *                    those levels' records through HBM;
 *   "rank_windows"   0 .. 64 (default 0: about 48 MB of ranks each): windows
 *                    of destination indices the rank scatter is split into;
 *   "ranges_per_cta" 1 .. 64 (default 4): radix-sort ranges per resident CTA;
 *   "blocks_per_sm"  1 .. 64 (default 16): flat-map / reduction blocks per SM.
 * The environment variable DOMAGG_TUNE="name=value,..." sets the defaults of
 * handles created afterwards.  Unknown names or values out of range return
 * DOMAGG_ERR_INVALID_ARG. */
domagg_status domagg_set_tuning(domagg_handle h, const char* name, int value);

/* Library version string ("checked build" when compiled with
 * DOMAGG_CHECKED: every kernel tests the indices it loads and stores
 * through, and an out-of-range one is reported as DOMAGG_ERR_BOUNDS by the
 * call's mid-call synchronisation or by domagg_sync_status). */
const char* domagg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DOMAGG_H */
