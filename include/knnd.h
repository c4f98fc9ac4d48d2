/*
 * knnd.h -- C ABI of the GB300 (sm_103a) K-nearest-neighbour descent library
 * for the Kullback-Leibler comparator on points of the probability simplex
 * (and, as variants, the reverse KL divergence, the squared Euclidean
 * distance and the inner product: knnd_params.comparator).
 *
 * Method: Baron & Darling, "Empirical complexity of comparator-based nearest
 * neighbor descent", arXiv:2202.00517.
 *   - problem statement (Sec. 2.1, Sec. 2.3): a set S of n objects and, for
 *     each x, a total order on S \ {x}; the output is the K-out digraph from
 *     each x to its K most similar objects;
 *   - comparator (Sec. 2.2, Sec. 4.4): y precedes z for x when
 *     D(x||y) < D(x||z), D(x||y) = sum_i x_i log(x_i / y_i); ties are broken
 *     by the smaller index (variants, Sec. 2 item (a): D(y||x), |x - y|^2);
 *   - initial graph (Sec. 3.2): every x picks K distinct friends uniformly;
 *   - one round (Sec. 3.1, Sec. 4.2): every x meets its co-friends, its
 *     friends' friends and its co-friends' friends; its new friend list is the
 *     K best of those and its old friends; all lists change together;
 *   - termination (Sec. 3.3): a sampled friend clustering rate; the build
 *     ends with the first round whose rate is no higher than the last one's.
 *
 * Conventions shared by every call:
 *   - Points: n rows of m coordinates, row-major with a leading dimension of
 *     `ld` elements (ld >= m), KNND_F32 or KNND_F64.  Every coordinate must be
 *     finite and, for the KL comparators, > 0 (points need not sum to
 *     exactly 1; they are used as stored).  Point pointers are DEVICE
 *     pointers unless a name says _host.
 *   - Graph: idx is n x K int32 (row x = x's friends), key is n x K float64
 *     (key[x][t] = D(x || idx[x][t]) evaluated in FP64 as
 *     sum_i x_i log x_i - sum_i x_i log y_i, both sums fma chains from 0;
 *     KNND_CMP_KL_REVERSE: D(idx[x][t] || x), the same with the roles
 *     swapped; KNND_CMP_SQEUCLIDEAN: (|x|^2 - 2 <x, y>) + |y|^2; KNND_CMP_INNER: 0 - <x, y>),
 *     newflag is n x K uint8 (1 when
 *     the entry was not in the row before the call).  Each row is sorted by
 *     (key ascending, idx ascending).  Caller-owned device buffers.
 *   - Work is enqueued on the handle's stream (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream).  Calls that return a host
 *     value synchronise that stream; the others are stream-ordered.
 *   - Scratch memory lives in the handle: it is allocated by knnd_create
 *     (the graph round loop's small state and its CUDA graph by the first
 *     knnd_build that uses them) and released by knnd_destroy.  Calls on one
 *     handle must not overlap.
 *   - Every call returns a knnd_status.  Arguments are validated on the host
 *     before any launch; on an error nothing is enqueued unless stated.
 *     No C++ exception crosses this interface.
 */
#ifndef KNND_H
#define KNND_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t knnd_status;
#define KNND_OK 0
#define KNND_EINVAL (-1)    /* bad argument: null pointer, shape or parameter out of range */
#define KNND_EDOMAIN (-2)   /* a coordinate is not finite, or (KL comparators) not > 0 (found on the device) */
#define KNND_ENOMEM (-3)    /* device allocation failed */
#define KNND_ECUDA (-4)     /* a CUDA runtime call or kernel launch failed */
#define KNND_ETIMEOUT (-5)  /* a bounded device wait ran out */
#define KNND_EOVERFLOW (-6) /* a size exceeds an internal limit */
#define KNND_ESTATE (-7)    /* call out of order (e.g. round before any prepare) */

typedef int32_t knnd_dtype;
#define KNND_F32 0
#define KNND_F64 1

/* How the join scores candidate pairs.  Every form returns the same graph:
 * the mixed forms filter with a rigorous FP32 error bound and re-score in
 * FP64 every candidate the bound cannot decide. */
typedef int32_t knnd_precision;
#define KNND_PREC_FP64 0        /* every pair scored in FP64 */
#define KNND_PREC_MIXED_FP32 1  /* FP32 CUDA-core filter + FP64 re-score */
#define KNND_PREC_MIXED_BF16X3 2 /* BF16 hi/lo split tiles on the tcgen05 tensor cores + FP64 re-score */
#define KNND_PREC_AUTO 3        /* the library chooses (currently MIXED_FP32) */

#define KNND_MAX_K 64
#define KNND_MAX_M 128
#define KNND_MAX_ROUNDS 64

/* Termination and debugging parameters (NULL -> the defaults shown). */
typedef struct {
    int32_t fcc_samples;          /* S, samples of the clustering rate per round (10000) */
    int32_t max_rounds;           /* cap on rounds, 1..KNND_MAX_ROUNDS (64) */
    int32_t stop_on_zero_updates; /* also stop after a round with no update (1) */
    int32_t debug;                /* 1: device bounds checks and error-bound audit; 2: as 1, and the
                                     tensor-core join's first tile of its first block issues no MMA,
                                     so its bounded wait runs out: the call reports KNND_ETIMEOUT
                                     (a test of the timeout path, with no fault) (0) */
    int32_t timing;               /* 1: CUDA events around every phase, see knnd_stats (0) */
    int32_t incremental;          /* 1: a round does not propose again a pair it met only through edges
                                     of the previous round's graph (0); see knnd_round */
    float stop_delta;             /* > 0: also stop after a round with fewer than stop_delta * n * K
                                     updates, Dong et al.'s delta-proportion rule (Sec. 2, Table 1) (0) */
    int32_t comparator;           /* KNND_CMP_*: how x ranks the other points (KNND_CMP_KL) */
    int32_t loop;                 /* KNND_LOOP_*: how knnd_build runs its rounds (KNND_LOOP_AUTO) */
    /* Execution choices that change the speed, never the result (0: the value the
     * committed tuning table gives for the shape's padded m and K): */
    int32_t split_den;            /* round 1 first runs the hubs [0, n / split_den) and merges them, so that
                                     the rest propose against tighter thresholds (2..64); 1: one phase */
    int32_t merge_keep;           /* candidates each lane of the merge's fast path keeps (4 or 8; K <= 32) */
    int32_t join_blocks;          /* resident 128-thread blocks per SM of the FP32 TMA join (1..8; at most
                                     what fits) */
    int32_t join_form;            /* KNND_JOIN_TMA or KNND_JOIN_PLAIN: how the FP32 filter gathers its rows
                                     (0: the tuning table's, TMA only from n >= 65536 on); the TMA form
                                     needs m <= 72 (padded to 8, 16, 24, 32, 48, 64 or 72 coordinates),
                                     K <= 32, no incremental proposals, not the inner product and, past
                                     32 padded coordinates, debug = 0; else plain loads are used */
} knnd_params;

/* The join kernel a build ran (knnd_build_info.join_kernel); the first two are
 * also the values of knnd_params.join_form. */
#define KNND_JOIN_TMA 1   /* FP32 filter, rows and columns gathered into shared memory by TMA */
#define KNND_JOIN_PLAIN 2 /* FP32 filter, rows gathered by plain loads */
#define KNND_JOIN_FP64 3  /* every pair in FP64 (precision FP64) */
#define KNND_JOIN_TC 4    /* BF16 hi/lo tiles on the tcgen05 tensor cores (precision MIXED_BF16X3) */

/* The round loop of knnd_build.  Both give the same graph and report. */
#define KNND_LOOP_AUTO 0  /* GRAPH, or HOST when timing = 1 */
#define KNND_LOOP_HOST 1  /* the host launches every round and reads the stop decision after it
                             (one stream synchronisation per round) */
#define KNND_LOOP_GRAPH 2 /* one CUDA-graph launch per build: a while node whose body is one round
                             and a one-thread kernel that applies the stop rule on the device and
                             sets the node's condition; one synchronisation per build.  The graph
                             is captured on the first build and kept for later builds with the same
                             idx, key and newflag pointers.  Not with timing = 1 (EINVAL) */

/* Comparators (Sec. 2 item (a): the comparator of x is any function of x that
 * ranks the other points; keys returned are the comparator's values). */
#define KNND_CMP_KL 0          /* D(x || y), the paper's (Sec. 2.2, Sec. 4.4); coordinates > 0 */
#define KNND_CMP_KL_REVERSE 1  /* D(y || x): the asymmetric divergence the other way round; coordinates > 0 */
#define KNND_CMP_SQEUCLIDEAN 2 /* |x - y|^2 = (|x|^2 - 2 <x, y>) + |y|^2 (fma chains): a symmetric metric
                                  comparator; any finite coordinates */
#define KNND_CMP_INNER 3       /* 0 - <x, y> (fma chain): maximum inner product neighbours, the largest
                                  inner products first (not a metric); any finite coordinates */

/* Why knnd_build stopped. */
#define KNND_STOP_FCC 1        /* clustering hits did not increase (Sec. 3.3 (iv)) */
#define KNND_STOP_ZERO 2       /* a round made no update */
#define KNND_STOP_MAX_ROUNDS 3 /* max_rounds reached */
#define KNND_STOP_DELTA 4      /* fewer than stop_delta * n * K updates (params.stop_delta) */

/* Per-build report, filled by knnd_build / knnd_build_host (host memory). */
typedef struct {
    int32_t rounds;                          /* rounds performed, the stopping one included */
    int32_t stop_reason;                     /* KNND_STOP_* */
    int64_t updates[KNND_MAX_ROUNDS];        /* updates[r-1]: new list entries made by round r */
    int64_t fcc_hits[KNND_MAX_ROUNDS + 1];   /* fcc_hits[r]: hits of the graph after round r */
    int64_t proposals;                       /* candidate pairs scored by the join, all rounds */
    int64_t init_pairs;                      /* pairs scored by the initial graph (n*K) */
    int64_t rescored;                        /* mixed forms: pairs re-scored in FP64 */
    int64_t bound_violations;                /* debug audit: low-precision errors above the bound (must be 0) */
    int64_t merge_fallbacks;                 /* rows the merge finished on its serial path */
    int64_t join_survivors;                  /* candidates the join passed to the merge, all rounds */
    int64_t bound_audited;                   /* debug audit: pairs whose low-precision dot was checked */
    int32_t join_kernel;                     /* KNND_JOIN_*: the join the rounds ran */
    int32_t reserved;
} knnd_build_info;

/* Phases of the descent, for the per-phase timing of knnd_stats. */
#define KNND_PHASE_PREPARE 0 /* log table, -H(x), FP32 copies */
#define KNND_PHASE_INIT 1    /* initial random K-out graph */
#define KNND_PHASE_CSR 2     /* co-friend lists (count, scan, fill) */
#define KNND_PHASE_JOIN 3    /* hub-centric local join */
#define KNND_PHASE_MERGE 4   /* bounded top-K update, update count */
#define KNND_PHASE_FCC 5     /* clustering-rate sample */
#define KNND_NUM_PHASES 6

/* Counters kept by a handle since its creation. */
typedef struct {
    int64_t kernel_launches;                  /* kernels this handle has launched */
    int64_t rounds;                           /* rounds run */
    int64_t workspace_bytes;                  /* device scratch held by the handle */
    int64_t phase_count[KNND_NUM_PHASES];     /* timed instances of each phase (timing = 1) */
    double phase_ms[KNND_NUM_PHASES];         /* their summed CUDA-event milliseconds */
} knnd_stats;

typedef struct knnd_handle knnd_handle;

/* Create a handle for n points of m coordinates and K friends per point
 * (2 <= K <= min(n-1, KNND_MAX_K), 1 <= m <= KNND_MAX_M, n < 2^31) and
 * allocate its scratch on the current CUDA device.  `stream` is the
 * cudaStream_t (as void*) all later calls enqueue on.
 * Errors: EINVAL (shape or parameter out of range, out == NULL), ENOMEM,
 * ECUDA.  On error *out is NULL. */
knnd_status knnd_create(knnd_handle **out, int64_t n, int32_t m, int32_t K, knnd_dtype dtype,
                        knnd_precision precision, const knnd_params *params, void *stream);

/* Release the handle and its scratch (synchronises its stream).  NULL is a no-op. */
void knnd_destroy(knnd_handle *h);

/* Replace the stream later calls enqueue on. */
knnd_status knnd_set_stream(knnd_handle *h, void *stream);

/* Precompute from the points (log table, -H(x), FP32 copies and the FP32
 * error-bound scale).  Reads n x m coordinates at `points` (device, row
 * stride ld elements).  Synchronises the stream to report EDOMAIN when a
 * coordinate is not finite or not > 0.  knnd_init_graph, knnd_round and
 * knnd_build call it themselves when given a non-NULL points pointer. */
knnd_status knnd_prepare(knnd_handle *h, const void *points, int64_t ld);

/* Initial random K-out graph (Sec. 3.2): every x draws K distinct friends
 * y != x from the Philox4x32-10 stream keyed by `seed` with counter
 * (x, 0, 0, block), each as y' = Lemire-uniform in [0, n-1), y = y' + (y' >= x),
 * a repeated value drawn again; rows are then sorted by (key, idx).
 * points: device points or NULL (reuse the prepared ones).
 * idx, key: out, n x K device.  newflag: out, n x K device or NULL (all 1).
 * Errors: EINVAL, ESTATE (points NULL and never prepared), EDOMAIN, ECUDA. */
knnd_status knnd_init_graph(knnd_handle *h, const void *points, int64_t ld, uint64_t seed, int32_t *idx,
                            double *key, uint8_t *newflag);

/* One synchronous round r >= 1 (Sec. 3.1, Sec. 4.2) from G_{r-1} to G_r, in
 * place: idx/key hold G_{r-1} on entry and G_r on return (device, n x K,
 * rows sorted by (key, idx)); newflag (device n x K or NULL) marks the
 * entries of G_r absent from G_{r-1}.  Pool of x: friends, co-friends,
 * friends of friends, friends of co-friends, minus x; G_r(x) = its K best.
 * Incremental proposals (params.incremental = 1 and newflag non-NULL):
 * newflag is also read on entry, as the flags of G_{r-1} that the previous
 * knnd_init_graph / knnd_round call wrote for this graph (all 1 for a graph
 * from elsewhere).  A pair the hub tiles meet only through edges whose flag
 * is 0 was in round r-1's pool already, so it is either in G_{r-1}(x) or
 * worse than its K-th entry, and is not proposed again: the result is the
 * same graph with fewer candidates to merge.  Every pair is still scored.
 * updates (device int64 or NULL) receives the number of new entries;
 * fcc_hits (device int64 or NULL) receives the clustering hits of G_r drawn
 * from stream (seed, counter (s, r, 1, block)) for s < fcc_samples
 * (Sec. 3.3).  points: device points or NULL (reuse the prepared ones).
 * Errors: EINVAL, ESTATE, EDOMAIN, ECUDA, EOVERFLOW (debug checks). */
knnd_status knnd_round(knnd_handle *h, const void *points, int64_t ld, uint64_t seed, int32_t round,
                       int32_t *idx, double *key, uint8_t *newflag, int64_t *updates, int64_t *fcc_hits);

/* Clustering hits (Sec. 3.3) of graph idx (device n x K) for round number
 * `round`: S samples drawn from stream (seed, counter (s, round, 1, block)):
 * x = uniform [0, n), i = uniform [0, K), j' = uniform [0, K-1),
 * j = j' + (j' >= i); a hit when idx[x][j] is a friend of idx[x][i] or the
 * reverse.  hits: device int64, overwritten.  Errors: EINVAL, ECUDA. */
knnd_status knnd_fcc(knnd_handle *h, const int32_t *idx, uint64_t seed, int32_t round, int64_t *hits);

/* Full build (Sec. 3): initial graph, then rounds until the clustering hits
 * of round r do not exceed those of round r-1, or (stop_on_zero_updates) a
 * round makes no update, or (stop_delta) too few updates, or max_rounds.
 * points: device (non-NULL).  idx, key: out, device n x K (G after the
 * stopping round).  newflag: device n x K or NULL.  info: host, filled.
 * Synchronises the stream once per round (KNND_LOOP_HOST) or once per build
 * (KNND_LOOP_GRAPH; the first build with new idx/key/newflag pointers also
 * captures and instantiates the round graph, which the handle then keeps).
 * Errors: EINVAL, EDOMAIN, ECUDA, EOVERFLOW, ENOMEM (loop state). */
knnd_status knnd_build(knnd_handle *h, const void *points, int64_t ld, uint64_t seed, int32_t *idx,
                       double *key, uint8_t *newflag, knnd_build_info *info);

/* knnd_build from and to HOST memory: copies the points in (one
 * cudaMemcpyAsync into handle-owned device memory), builds, and copies idx
 * and key out; returns after the copies complete.  points_host: n x m with
 * row stride ld; idx_host (n x K int32), key_host (n x K float64): host
 * outputs (pinned memory gives full copy bandwidth).  Errors: as knnd_build. */
knnd_status knnd_build_host(knnd_handle *h, const void *points_host, int64_t ld, uint64_t seed,
                            int32_t *idx_host, double *key_host, knnd_build_info *info);

/* Largest sample count knnd_fcc_noalloc accepts. */
#define KNND_NOALLOC_MAX_SAMPLES (1 << 20)

/* The clustering sample of knnd_fcc without a handle and without allocating
 * any device memory.  The paper has no counterpart: this entry point serves
 * callers that cannot call cudaMalloc -- an application whose memory pool or
 * caching allocator already holds nearly all device memory, a serving loop
 * that forbids allocation after start-up, a plug-in whose host requires all
 * allocations to go through the host's allocator -- and so cannot create a
 * handle, but run their own descent loop and need the stop test.
 * Same draws and hit rule as knnd_fcc: idx (device, n x K int32), samples S
 * in [1, KNND_NOALLOC_MAX_SAMPLES] (EOVERFLOW above it), hits (device int64,
 * overwritten).  On a graph whose indices all lie in [0, n) the count equals
 * knnd_fcc's.  When a sampled friend index lies outside [0, n) the two
 * differ: knnd_fcc counts that sample as a miss and records the bad index in
 * the handle's sticky status (knnd_sync returns EINVAL), while this call
 * writes -1 to hits.  Enqueued on `stream` (cudaStream_t as void*).
 * Scratch: a fixed array of about 32 KB in the library's device memory,
 * loaded with the library and held by every GPU that loads it until the
 * process exits.  Every call looks up that array's device address in the
 * current context (cudaGetSymbolAddress, with the device current; a host-side
 * query, not a stream operation); the first call on a device also loads the
 * library's device code there, so make that first call before any stream
 * capture.  All calls on a device share the array, and each call clears its
 * error word before sampling: calls that overlap on the GPU race.  Allocates
 * nothing, frees nothing.
 * Errors: EINVAL (null pointer, shape as in knnd_create), EOVERFLOW, ECUDA. */
knnd_status knnd_fcc_noalloc(const int32_t *idx, int64_t n, int32_t K, uint64_t seed, int32_t round,
                             int32_t samples, int64_t *hits, void *stream);

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11), the counter-based generator behind every random
 * draw of this library: the uniform choices of the initial graph (Sec. 3.2)
 * and of the clustering sample (Sec. 3.3) use counter (c0, c1, c2, block) and
 * key (low and high 32 bits of the seed).  For i < count, out[4i .. 4i+3] =
 * the ten-round Philox bijection of the counter ctr_key[6i .. 6i+3] under the
 * key ctr_key[6i+4 .. 6i+5], computed by the same device routine the draws
 * use; it exists so that this routine can be checked against the generator's
 * published known-answer vectors.  ctr_key: device uint32, count x 6; out:
 * device uint32, count x 4; enqueued on `stream` (cudaStream_t as void*).
 * Errors: EINVAL (null pointer with count > 0, count < 0 or >= 2^31), ECUDA. */
knnd_status knnd_philox4x32_10(const uint32_t *ctr_key, uint32_t *out, int64_t count, void *stream);

/* Measurement support for the roofline fractions the benchmark reports (not
 * part of the method): the rate of one FMA pipe on the current device.  Runs
 * blocks_per_sm blocks of 256 threads on every SM, each thread eight
 * independent fma chains of `iters` steps: kind 0 FP32 fma (the join's filter
 * arithmetic), 1 packed two-wide FP32 fma (FFMA2, the TMA join's form), 2 FP64
 * fma (the FP64 form and the re-scores).  sink: device, >= 3 floats, all 0 on
 * entry (operands the compiler cannot fold).  Returns the FLOPs executed
 * (2 per fma, 4 per packed fma) in *flops and the CUDA-event milliseconds of the
 * launch in *ms; synchronises `stream`.  Changes no device setting.
 * Errors: EINVAL (kind, blocks_per_sm outside 1..64, iters < 1, null pointer), ECUDA. */
knnd_status knnd_fma_peak(int32_t kind, int32_t blocks_per_sm, int64_t iters, float *sink, double *flops,
                          float *ms, void *stream);

/* Synchronise the handle's stream and return (and clear) the sticky device
 * status: EDOMAIN (bad coordinate), EINVAL (a graph index outside [0, n)
 * met by a kernel, which skipped it), EOVERFLOW (debug bucket check), or OK.
 * Kernels never access memory out of bounds on bad input; they record it
 * here instead. */
knnd_status knnd_sync(knnd_handle *h);

/* ---- batched form --------------------------------------------------------
 * Many independent instances built together (the same method, per instance,
 * as knnd_build).  Instances with equal (m, K) share kernel launches: each
 * phase is one launch over all of them; a class too large for the workspace
 * budget is cut into sub-batches.  Each sub-batch runs as one CUDA graph
 * (captured at the first knnd_batch_run and kept): its rounds are a
 * conditional while loop whose stop test runs on the device, per instance.
 * Sub-batches run on up to four internal streams at once, each with its own
 * workspace.  Every instance gets the graph, rounds and counts a separate
 * knnd_build with its seed would give. */
typedef struct {
    const void *points; /* device: n x m, row stride ld elements, dtype of the call */
    int64_t ld;
    int64_t n;          /* 3 <= n < 2^31 */
    int32_t m;          /* 1 <= m <= KNND_MAX_M */
    int32_t K;          /* 2 <= K <= min(n-1, KNND_MAX_K) */
    uint64_t seed;
    int32_t *idx;       /* out: device n x K, indices local to the instance */
    double *key;        /* out: device n x K */
} knnd_instance;

typedef struct knnd_batch knnd_batch;

/* Plan the sub-batches of `count` instances (the array is copied; the points
 * and output pointers must stay valid until the batch is destroyed) and
 * allocate the workspaces.  workspace_limit: device bytes one sub-batch may
 * plan for (<= 0: 32 GiB); up to four workspaces, each the size of the largest
 * sub-batch given to it, as many as 85 % of the free device memory holds.
 * Errors: EINVAL (a bad instance or parameter), ENOMEM, ECUDA. */
knnd_status knnd_batch_create(knnd_batch **out, int32_t count, const knnd_instance *inst, knnd_dtype dtype,
                              knnd_precision precision, const knnd_params *params, int64_t workspace_limit,
                              void *stream);

/* Build every instance (Sec. 3: initial graph, rounds to the statistical
 * stop, per instance).  The work starts after what is already enqueued on the
 * batch's stream, and the stream waits for it; the call returns when every
 * instance is built (no synchronisation inside a sub-batch).  info: host
 * array of `count` reports, or NULL.  A bad coordinate (EDOMAIN) or index
 * (EINVAL) met on the device is reported once every sub-batch has run; the
 * outputs are then unspecified.  Errors: EDOMAIN, EINVAL, ECUDA. */
knnd_status knnd_batch_run(knnd_batch *b, knnd_build_info *info);

/* Sub-batches planned, workspace bytes, kernels launched so far (each NULL-able). */
knnd_status knnd_batch_info(const knnd_batch *b, int32_t *sub_batches, int64_t *workspace_bytes,
                            int64_t *kernel_launches);

/* Release the batch and its workspace (synchronises its stream).  NULL is a no-op. */
void knnd_batch_destroy(knnd_batch *b);

/* knnd_batch_create + knnd_batch_run + knnd_batch_destroy. */
knnd_status knnd_build_batched(int32_t count, const knnd_instance *inst, knnd_dtype dtype,
                               knnd_precision precision, const knnd_params *params, int64_t workspace_limit,
                               knnd_build_info *info, void *stream);

/* Counters of the handle (host struct).  Synchronises the stream when
 * timing is on, to read the pending phase events. */
knnd_status knnd_get_stats(knnd_handle *h, knnd_stats *stats);

/* Zero the phase timings and launch counters of knnd_stats. */
knnd_status knnd_reset_stats(knnd_handle *h);

/* Static text for a status code. */
const char *knnd_status_string(knnd_status s);

/* Library version, major*10000 + minor*100 + patch. */
int32_t knnd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KNND_H */
