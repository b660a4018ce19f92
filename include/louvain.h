/*
 * louvain.h -- C ABI of the GB300 (sm_103a) Louvain library.
 *
 * The library runs the data-parallel hot path of the Louvain method as
 * studied in arXiv 2501.19004 ("CPU vs. GPU for Community Detection:
 * Performance Insights from GVE-Louvain and nu-Louvain"): the local-moving
 * phase (Sec. 4.2.2, Algorithm 2 / Algorithm 5), the aggregation phase
 * (Sec. 4.2.3, Algorithm 3 / Algorithm 6) and the pass loop around them
 * (Sec. 4.2.1, Algorithm 1 / Algorithm 4), with modularity as defined by
 * Eq. 1 and delta-modularity by Eq. 2 (Sec. 3.2).
 *
 * Schedule.  The paper moves vertices asynchronously; this library fixes one
 * deterministic semi-synchronous schedule so that every run is reproducible:
 * in iteration t of pass p, vertex i belongs to bucket
 *     fmix32(i ^ fmix32(fold(seed) ^ (((p << 8) | t) * 0x9E3779B1))) mod B
 * (fmix32 = the MurmurHash3 finaliser, fold(s) = low32(s) ^ high32(s)).
 * Bucket by bucket, the unprocessed vertices of the bucket are marked
 * processed, each picks the neighbouring community c maximising
 *     s(c) = 2m K_{i->c} - K_i Sigma_c            (= 2m^2 dQ + const, Eq. 2)
 * against a snapshot of the memberships and community weights (ties go to
 * the lowest id), moves if s(c*) > 2m K_{i->d} - K_i (Sigma_d - K_i) and
 * Pick-Less mode (Sec. 4.3.1) does not forbid c* > d, and then all moves of
 * the bucket are applied and the neighbours of movers are marked
 * unprocessed (vertex pruning, Sec. 4.1.6).  An iteration ends the phase when
 * 2 * sum(gains) / (2m)^2 <= tau.  All of this is exact integer arithmetic.
 * louvain_config.asynchronous = 1 selects the paper's own asynchronous form
 * instead (moves applied in place as they are decided; not reproducible).
 * louvain_config.refine = 1 selects the Leiden form (Traag, Waltman and van
 * Eck 2019, which Sec. 5.2 and Sec. 6 expect the paper's findings to extend
 * to): each pass's partition is refined, deterministically, before it is
 * aggregated (see the field).
 *
 * Conventions for every function below:
 *   - A status code is returned; nothing aborts, exits or traps.  On error,
 *     louvain_last_error() describes the failure.
 *   - Arrays passed in are borrowed for the duration of the call (device
 *     graphs: until louvain_destroy).  Outputs are caller-owned.
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL means
 *     the legacy default stream.
 */
#ifndef LOUVAIN_GB300_H
#define LOUVAIN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct louvain_ctx louvain_ctx; /* opaque, library-owned */

typedef enum {
  LOUVAIN_OK = 0,
  LOUVAIN_E_INVAL = 1,          /* bad argument or malformed CSR */
  LOUVAIN_E_NOMEM = 2,          /* device or host allocation failed */
  LOUVAIN_E_CUDA = 3,           /* a CUDA call failed (see louvain_last_error) */
  LOUVAIN_E_HASH_OVERFLOW = 4,  /* a hashtable probe sequence exceeded its bound
                                   (the paper's "failed" result of Algorithm 7, after
                                   MAX_RETRIES probes).  Tables hold at least twice as
                                   many slots as keys, so the bound is the table size
                                   and no input reaches it; a library built with
                                   -DLOUVAIN_MAX_PROBES=k gives up after k probes.
                                   A failed run leaves the context usable. */
  LOUVAIN_E_TIMEOUT = 5,        /* a bounded device-side wait gave up (reserved: no
                                   kernel of this library waits on a flag) */
  LOUVAIN_E_OVERFLOW = 6,       /* 2m >= 2^32: scores would not fit in int64 */
  LOUVAIN_E_STATE = 7           /* call out of order (e.g. memberships before run) */
} louvain_status;

/* Undirected weighted graph in CSR form (Sec. 3: G(V, E, w) with w_ij = w_ji;
 * Table 2 counts both directions of every edge, and so does nnz).
 *   offsets [n+1] int64, offsets[0] = 0, non-decreasing, offsets[n] = nnz
 *   cols    [nnz] int32, 0 <= cols[k] < n; a self-loop is stored once
 *   weights [nnz] int32 > 0, or NULL for unit weights
 * on_device = 1: device pointers, borrowed until louvain_destroy;
 * on_device = 0: host pointers, copied to the device by louvain_create. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int64_t *offsets;
  const int32_t *cols;
  const int32_t *weights;
  int32_t on_device;
} louvain_graph;

typedef enum { LOUVAIN_MODE_PLAIN = 0, LOUVAIN_MODE_LEARNED = 1 } louvain_mode;

/* Run parameters.  Defaults (louvain_config_default) are the paper's:
 * MAX_PASSES 10 and MAX_ITERATIONS 20 (Sec. 4.3 item 2, Sec. 4.1.2),
 * tau = 0.01 (Sec. 4.1.4), TOLERANCE_DROP 10 (Sec. 4.1.3), tau_agg 0.8
 * (Sec. 4.1.5), Pick-Less every rho = 4 iterations (Sec. 4.3.1). */
typedef struct {
  int32_t max_passes;
  int32_t max_iterations;        /* 1 .. 255 */
  double tolerance;
  double tolerance_drop;
  double aggregation_tolerance;
  int32_t pickless_period;       /* rho; 0 disables Pick-Less mode */
  int32_t buckets;               /* B of the deterministic schedule, 1 .. 65536 (4) */
  uint64_t schedule_seed;
  int32_t mode;                  /* louvain_mode */
  const float *model;            /* LEARNED: host pointer to the predictor's
                                    parameters (louvain_model_size floats) */
  float skip_threshold;          /* LEARNED: skip a vertex when p < threshold */
  int32_t record_pass_modularity;/* 1: compute Q after every pass (stats) */
  int32_t check_symmetry;        /* 1: louvain_create verifies w_ij = w_ji (host graphs) */
  uint32_t profile_mask;         /* bit k: time kernel group k with CUDA events
                                    (ids in louvain_stats' "kernels"); 0 = off */
  int64_t trace_capacity;        /* > 0: record up to this many (features, moved)
                                    samples of evaluated vertices (louvain_traces) */
  float trace_rate;              /* fraction of decisions recorded (hash-sampled) */
  int32_t learned_fallback;      /* LEARNED: after the learned iterations of a pass,
                                    plain iterations (no skipping) run:
                                    0: over the flagged vertices (every skipped
                                       vertex kept its flag) until an iteration's
                                       dQ <= tau (the plain rule);
                                    1: first over all vertices, until an iteration
                                       makes no move;
                                    2: first over all vertices, until dQ <= tau;
                                    3: none; instead, when a learned iteration's
                                       dQ <= tau, the vertices the predictor
                                       skipped in it are evaluated at once (its
                                       completion step, same iteration), and the
                                       phase ends only if the iteration's dQ,
                                       completion included, is still <= tau */
  int32_t learned_skip_clears;   /* LEARNED: 1 = a skip counts as a decision to stay
                                    and clears the vertex's flag (it returns when a
                                    neighbour moves); 0 = skipped vertices keep
                                    their flag */
  int64_t table_window;          /* the global hashtables of hub vertices (degree above
                                    32768) and large communities (members holding more
                                    than 8192 entries) are processed in rounds of this
                                    many 8-byte slots (at least the largest table);
                                    0 = half of the pass's bound on their total size.
                                    Results do not depend on it. */
  int32_t asynchronous;          /* 1: the asynchronous form of the paper's GPU
                                    algorithm (Algorithm 5 as written, Sec. 4.3):
                                    each iteration is one sweep over all unprocessed
                                    vertices, and every move is applied the moment
                                    it is decided (C'[i] and Sigma' by atomics), so
                                    later decisions of the sweep see it.  Results
                                    then depend on thread timing and are not
                                    reproducible; buckets and schedule_seed are
                                    ignored.  Plain mode, no traces, single graphs
                                    only (LOUVAIN_E_INVAL otherwise).  0: the
                                    deterministic bucket schedule. */
  int32_t learned_min_degree;    /* LEARNED and trace recording: only vertices of at
                                    least this degree are candidates of the predictor
                                    and keep features (and only they are recorded);
                                    lower-degree vertices are always evaluated when
                                    flagged, as in the plain method.  0 = all. */
  int32_t refine;                /* 1: the Leiden form (Traag, Waltman and van Eck
                                    2019, which Sec. 5.2 and Sec. 6 of the paper
                                    expect its findings to extend to): after local
                                    moving, the partition P is refined and the
                                    refined partition is aggregated; the next pass
                                    starts every super-vertex in its community of P.
                                    Refinement: one sweep over 4B buckets of
                                    (vertex, pass, iteration 255), the hash of the
                                    schedule with 4B in place of B (fewer
                                    simultaneous decisions than local moving); a
                                    vertex that is
                                    still a singleton of the refined partition and
                                    well connected to its community C of P
                                    (2m K_{i->C} >= K_i (Sigma_C - K_i), K_{i->C}
                                    without the self-loop) joins the refined
                                    community inside C with the largest score
                                    2m K_{i->T} - K_i Sigma_T (lowest id on ties)
                                    if that score is positive; a vertex that any
                                    decision of the bucket chose as its target stays
                                    and stops being a singleton.  The low-shrink test
                                    compares the refined communities with n'; the
                                    memberships are P's.  PLAIN mode, deterministic
                                    schedule, single graphs only, and not with
                                    louvain_run_passes (LOUVAIN_E_INVAL otherwise).
                                    0: the Louvain form. */
} louvain_config;

/* Fill `cfg` with the defaults above (mode PLAIN, seed 0). */
void louvain_config_default(louvain_config *cfg);

/* Validate the graph (offsets monotone, ids in range, weights > 0,
 * optional symmetry), copy or borrow it, and allocate all device workspace
 * (stream-ordered on `stream`).  Returns LOUVAIN_E_OVERFLOW if the total
 * weight 2m is 2^32 or more.  *out receives the context. */
louvain_status louvain_create(const louvain_graph *graph, const louvain_config *cfg, void *stream,
                              louvain_ctx **out);

/* Run the whole method (all passes and the final modularity) on the
 * context's stream; returns when the result is ready. */
louvain_status louvain_run(louvain_ctx *ctx);

/* Pass-level control and checkpoints of a single-graph run (Algorithm 1's
 * pass loop; a pass is one local-moving phase plus one aggregation).
 *
 * louvain_run_passes starts a run like louvain_run but, when
 * max_new_passes > 0 and the run still has a pass to do after that many
 * passes, stops between two passes: *suspended = 1 (may be NULL), and the
 * context holds the dendrogram, the super-vertex graph, its vertex weights,
 * the tolerance of the next pass and the records of the passes done.
 * Otherwise the run finishes (*suspended = 0) exactly as louvain_run.
 * louvain_resume continues a suspended run the same way (max_new_passes <= 0:
 * to the end); LOUVAIN_E_STATE if the context is not suspended.  A suspended
 * run gives no results yet (LOUVAIN_E_STATE from louvain_modularity and the
 * other result calls).  Stopping and resuming never changes results: the
 * memberships, the exact modularity and the per-pass and per-iteration
 * records equal those of an uninterrupted run.  louvain_stats then times
 * only the passes run in this context since the last start or load.
 * Batched contexts: LOUVAIN_E_INVAL. */
louvain_status louvain_run_passes(louvain_ctx *ctx, int32_t max_new_passes, int32_t *suspended);
louvain_status louvain_resume(louvain_ctx *ctx, int32_t max_new_passes, int32_t *suspended);

/* Checkpoint of a suspended run into a caller-owned host buffer (8-byte
 * aligned, at least *size bytes; buf = NULL only reports *size).  Layout,
 * native byte order: a header of 20 int64 words (magic "LVCKPT01", sizes, an
 * FNV-1a checksum of the payload, the input graph's n, nnz, 2m and weight
 * kind, a fingerprint of every setting that decides results, the next pass,
 * tau and the run totals), then the records of the passes done, C[n] int32,
 * K[n'] int64 and the super-vertex graph as a compact CSR (offsets[n'+1]
 * int64, cols[nnz'] int32, weights[nnz'] uint32).  LOUVAIN_E_STATE if the
 * context is not suspended; LOUVAIN_E_INVAL for a short or unaligned buffer. */
louvain_status louvain_save_state(const louvain_ctx *ctx, void *buf, size_t cap, size_t *size);

/* Restore a checkpoint into a context created on the same input graph with
 * the same result-deciding settings (and model, in learned mode); the
 * context is then suspended and louvain_resume continues the run.  Any
 * previous results of the context are dropped, also when the checkpoint is
 * refused.  It is refused (LOUVAIN_E_INVAL, nothing suspended; the context
 * stays usable for louvain_run) when its magic, size or checksum is
 * wrong, when it was taken on another graph or configuration, or when its
 * rows, dendrogram ids, vertex weights or entries are out of range (entries
 * are checked on the device: columns in [0, n'), weights > 0, their sum
 * 2m).  Recorded traces are not part of a checkpoint. */
louvain_status louvain_load_state(louvain_ctx *ctx, const void *buf, size_t size);

/* Final modularity Q (Eq. 1) of the last run, as a double, and optionally
 * its exact numerator 2m*S_in - sum_c Sigma_c^2 and denominator (2m)^2 as
 * (hi, lo) pairs of a 128-bit integer (either pointer may be NULL). */
louvain_status louvain_modularity(const louvain_ctx *ctx, double *q, int64_t *num_hi_lo,
                                  int64_t *den_hi_lo);

/* Final community of every input vertex, dense ids in [0, |Gamma|) ordered
 * like the first-level ids.  `out` is caller-owned [n], host or device. */
louvain_status louvain_memberships(const louvain_ctx *ctx, int32_t *out, int32_t out_on_device);

/* Per-iteration and per-pass records of the last run, same layout as the CPU
 * oracle's: iter_stats[max_passes][max_iterations][4] = (vertices evaluated,
 * moves, gain_hi, gain_lo); pass_stats[max_passes][6] = (n', nnz', l_i,
 * |Gamma|, Qnum_hi, Qnum_lo); summary[8] = (passes, |Gamma|, Qnum hi/lo,
 * Qden hi/lo, 2m, exit reason 0 max passes / 1 converged / 2 low shrink).
 * Any pointer may be NULL. */
louvain_status louvain_records(const louvain_ctx *ctx, int64_t *iter_stats, int64_t *pass_stats,
                               int64_t *summary);

/* JSON object with timings per phase and per pass (CUDA events), counts and
 * the memory footprint.  Returns LOUVAIN_E_INVAL if `cap` is too small. */
louvain_status louvain_stats(const louvain_ctx *ctx, char *json, size_t cap);

/* Change which kernel groups the next runs time with CUDA events (the
 * profile_mask of louvain_config).  Timing adds two event records per timed
 * launch and nothing else. */
louvain_status louvain_set_profile(louvain_ctx *ctx, uint32_t profile_mask);

/* ---- Launch schedule and autotuner (an addition of this library; the paper
 * fixes one kernel configuration).  A schedule is louvain_schedule_words()
 * int32 words:
 *   [0] group_max: largest degree handled by 8-lane groups (16 .. 64;
 *       16 = no 8-lane groups); [1] half_max: largest degree handled by
 *       16-lane groups (group_max .. 128; = group_max for none); [2]
 *       warp_max: largest degree handled by a warp (half_max .. 256; larger
 *       degrees up to 1024 go to 128-thread blocks);
 *   [3..11] blocks per SM of the local-moving kernels of the thread, warp,
 *       128-thread, 512-thread, hub (<= 3), 8-lane group, wide (degrees
 *       4097 .. 32768; its kernel runs one block per SM from a work queue and
 *       ignores this word), a reserved word, and 16-lane group bins (1 .. 64);
 *   [12..18] blocks per SM of the aggregation kernels of the thread, warp,
 *       128-thread, 512-thread, big-community (<= 3), 1024-thread and group
 *       bins;
 *   [19] graphs: 1 = each local-moving iteration is replayed from a CUDA
 *       graph captured once per pass (plain mode, no profiling);
 *   [20] concurrent: 1 = a bucket's bin kernels (and an aggregation's) run at
 *       the same time on side streams of the context.
 * Results of the deterministic form never depend on the schedule: every bin
 * computes the same exact decisions.  The schedule belongs to the context
 * and is used by its next runs. */
int32_t louvain_schedule_words(void);
louvain_status louvain_get_schedule(const louvain_ctx *ctx, int32_t *words, int32_t n);
louvain_status louvain_set_schedule(louvain_ctx *ctx, const int32_t *words, int32_t n);

/* Choose the context's schedule by timed runs of its own graph (at most
 * max_runs trials; a whole-run trial is the faster of two runs), in order:
 * the bin thresholds by whole-run time (a triple replaces the current one
 * only if it is at least 1.5% faster, more than run-to-run noise); the
 * blocks per SM of every bin by per-kernel CUDA-event time (the current
 * values are one of the candidates); concurrent bin kernels on or off;
 * graph replay on or off.  The tuned schedule is kept only if it beats the
 * starting one.  json (may be NULL) receives {"runs", "start_ms", "tuned_ms", "schedule",
 * "trials"}.  The context holds a valid result of the chosen schedule
 * afterwards. */
louvain_status louvain_autotune(louvain_ctx *ctx, int32_t max_runs, char *json, size_t cap);

/* Release all device memory of the context (stream-ordered). */
void louvain_destroy(louvain_ctx *ctx);

/* Description of the last error on this context (or of the last failed
 * louvain_create when ctx is NULL).  Never NULL. */
const char *louvain_last_error(const louvain_ctx *ctx);

/* Modularity (Eq. 1) of an arbitrary membership on a graph, computed on the
 * device.  graph and membership are both device or both host arrays
 * (graph->on_device); membership ids lie in [0, n) (LOUVAIN_E_INVAL
 * otherwise; nothing is written for such a vertex).  q and the exact
 * numerator/denominator (hi, lo) as in louvain_modularity. */
louvain_status louvain_modularity_of(const louvain_graph *graph, const int32_t *membership, void *stream,
                                     double *q, int64_t *num_hi_lo, int64_t *den_hi_lo);

/* ---- Learned vertex-activity predictor (an addition of this library; the
 * paper has no counterpart).  An 8 -> 32 -> 32 -> 1 MLP decides which
 * flagged vertices of a bucket the local-moving phase evaluates: a vertex
 * whose predicted probability of moving is below skip_threshold keeps its
 * flag and is skipped for this iteration.  After the learned iterations of a
 * pass converge, plain iterations without skipping follow: by default over
 * the flagged vertices (which include every skipped one) until the plain
 * method's tolerance test holds; learned_fallback selects a full sweep over
 * all vertices first, and a zero-move stopping rule.  These sweeps bound the
 * modularity gap to the plain method.  Parameters: W1[8][32], b1[32],
 * W2[32][32], b2[32], w3[32], b3 (fp32; W[k][n] maps input k to output n);
 * evaluation rounds x, W1, W2, w3 and the hidden ReLU outputs to bf16 and
 * accumulates in fp32 on the tensor cores.  Features per vertex, in order:
 * log2(1 + degree)/24, intra-community weight fraction and best-dQ margin
 * (s(c*) - s(d))/(2m K_i) at its last evaluation, moved at its last
 * evaluation, iteration/MAX_ITERATIONS, pass/MAX_PASSES, Sigma of its
 * community/2m, and the fraction of its sampled neighbours that moved since
 * its last evaluation (the whole row up to 96 entries; for longer rows the
 * neighbours j with fmix32(j ^ fmix32(i ^ 0x5BD1E995)) < 2^32 * 32 / degree,
 * or the whole row if more than 96 qualify).  Only vertices of degree at least learned_min_degree are
 * candidates; with learned_fallback = 3 an iteration that meets the
 * tolerance is completed by evaluating what it skipped (see below).
 */

/* louvain_modularity_of without any allocation, for callers that cannot let
 * a library allocate device memory (for example an application whose own
 * pool allocator owns the whole device, or a serving loop that must not call
 * cudaMalloc).  The paper has no counterpart.  Same result as
 * louvain_modularity_of; the graph and the membership must be device arrays
 * (graph->on_device = 1) and n may not exceed 1,048,576 (LOUVAIN_E_INVAL
 * beyond that).  Scratch lives in a fixed 8 MiB array inside the library
 * that every GPU loading the library keeps until exit; calls share it, so
 * calls that overlap on the GPU race.  The first call on a device does the
 * set-up: it loads the library's device code there, which reserves the
 * array; make it before your own pool claims the device's memory.  Every
 * call looks the array's address up again (no allocation once the code is
 * loaded), so a call after cudaDeviceReset of the device does that set-up
 * again.  The CSR is checked on the device before any entry
 * is read: offsets[0] = 0, offsets[n] = nnz, every row within [0, nnz) and
 * not decreasing, columns and membership ids in [0, n), weights > 0
 * (LOUVAIN_E_INVAL otherwise); 2m >= 2^32 gives LOUVAIN_E_OVERFLOW. */
louvain_status louvain_modularity_noalloc(const louvain_graph *graph, const int32_t *membership, void *stream,
                                          double *q, int64_t *num_hi_lo, int64_t *den_hi_lo);

/* ---- Batched runs: many independent graphs in one context.  The paper runs
 * one graph at a time and names the small, shrinking graphs of late passes
 * as the cause of nu-Louvain's lost parallelism (Sec. 5.2); a batch runs all graphs'
 * passes together, so every launch covers the vertices of every graph still
 * running.  Each graph gets exactly the result of its own run with the same
 * config: its own 2m (Eq. 2), its own iteration tolerance test, convergence
 * test (l_i <= 1) and aggregation tolerance test (Sec. 4.1.4, 4.1.5), and the
 * bucket schedule over its local vertex ids.
 *
 * `graph` is the union: graph g owns the vertices [vertex_offsets[g],
 * vertex_offsets[g+1]) (host array of num_graphs + 1 int64, 0 first, n last,
 * non-decreasing; empty graphs allowed), columns are union ids, and no entry
 * may leave its graph (LOUVAIN_E_INVAL).  Each graph's 2m must be below 2^32
 * (LOUVAIN_E_OVERFLOW); the union's may be larger.  The config must be the
 * plain mode without traces.  louvain_run runs the batch, louvain_memberships
 * returns, for every union vertex, its community's dense id within its own
 * graph, and louvain_modularity is refused (LOUVAIN_E_INVAL): per-graph
 * results come from louvain_batch_results. */
louvain_status louvain_create_batched(const louvain_graph *graph, const int64_t *vertex_offsets, int64_t num_graphs,
                                      const louvain_config *cfg, void *stream, louvain_ctx **out);

/* Per-graph results of the last batched run (host arrays, any may be NULL):
 * results[num_graphs][8] in the layout of louvain_records' summary (passes,
 * |Gamma|, Qnum hi/lo, Qden hi/lo, 2m, exit reason); q[num_graphs];
 * pass_records[num_graphs][max_passes][3] = (n', l_i, |Gamma|) of each pass
 * the graph ran.  LOUVAIN_E_INVAL on a context that is not batched. */
louvain_status louvain_batch_results(const louvain_ctx *ctx, int64_t *results, double *q, int64_t *pass_records);

/* Number of floats of the learned predictor's parameters (8->32->32->1 MLP). */
int64_t louvain_model_size(void);

/* Recorded samples of the last run (config.trace_capacity > 0): features
 * [count][8] and labels [count] (1 = the vertex moved when evaluated).  The
 * outputs are caller-owned, host or device (on_device); *count receives the
 * number of samples (at most cap). */
louvain_status louvain_traces(const louvain_ctx *ctx, float *features, float *labels, int64_t cap, int64_t *count,
                              int32_t on_device);

/* The predictor's arithmetic (the definition both louvain_mlp_forward and
 * louvain_mlp_gradient compute; bf() = round to the nearest bfloat16, ties
 * to even; every sum is accumulated in fp32 unless marked otherwise):
 *   forward, per row:  x~ = bf(x), W1~ = bf(W1), W2~ = bf(W2), w3~ = bf(w3);
 *     z1 = x~ W1~ + b1;   h1 = bf(max(z1, 0));
 *     z2 = h1 W2~ + b2;   h2 = bf(max(z2, 0));
 *     logit = h2 . w3~ + b3;   p = sigmoid(logit).
 *   backward of L = (1/n) sum_rows BCE(p, y):
 *     dl = (p - y) / n                                  (fp32, not rounded)
 *     db3 = sum dl;   dw3 = sum dl h2
 *     dz2 = dl w3~ [z2 > 0];   db2 = sum dz2            (dz2 not rounded)
 *     dW2 = h1^T bf(dz2)                                (bf16 operands)
 *     dh1 = bf(dz2) W2~^T;   dz1 = dh1 [z1 > 0];   db1 = sum dz1
 *     dW1 = x~^T bf(dz1)                                (bf16 operands)
 * So exactly two deltas are rounded, bf(dz2) and bf(dz1), each where it
 * enters a tensor-core contraction; bias and w3 gradients use the unrounded
 * fp32 deltas.  The fp32 sums run over the rows in tiles (16 rows per mma
 * step, 128 rows per block, block partials added in block order). */

/* Logits of n feature rows X[n][8] (device pointers; params on the device). */
louvain_status louvain_mlp_forward(const float *params, const float *X, int64_t n, float *logits, void *stream);

/* Gradient of the mean binary cross-entropy of sigmoid(logit) against
 * labels Y over n rows (the backward definition above), added into
 * grad[louvain_model_size()]; the mean loss is added into *loss (device
 * pointers; loss may be NULL). */
louvain_status louvain_mlp_gradient(const float *params, const float *X, const float *Y, int64_t n, float *grad,
                                    float *loss, void *stream);

/* Adam training of params (device, in/out) on (X, Y) (device): `epochs`
 * passes of minibatches of `batch` rows in a seeded order; per-epoch mean
 * losses into losses[epochs] (host, may be NULL). */
louvain_status louvain_mlp_train(float *params, const float *X, const float *Y, int64_t n, int32_t epochs,
                                 int32_t batch, float lr, uint64_t seed, float *losses, void *stream);

/* Library build description (architecture, version). */
const char *louvain_version(void);

#ifdef __cplusplus
}
#endif
#endif
