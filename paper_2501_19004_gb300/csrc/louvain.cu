// Host driver and C ABI of the GB300 Louvain library (include/louvain.h).
//
// The pass loop follows Algorithm 1 / Algorithm 4 of arXiv 2501.19004
// (Sec. 4.2.1 and the Appendix): per pass, vertex weights and identity
// memberships (pass_init), the local-moving phase (move.cu, Algorithm 5)
// until the iteration tolerance is met, the convergence and aggregation
// tolerance tests, renumbering, dendrogram lookup and aggregation (aggr.cu,
// Algorithm 6), then threshold scaling.  Everything stays on the device; the
// host only reads a few scalars per iteration (the exact gain sum) and per
// pass (community count, sizes).  The same loop can stop between two passes
// and resume, also from a checkpoint in host memory; a batch of graphs runs
// it in lockstep over their union (batch.cu); and louvain_autotune picks the
// launch schedule by timed runs.
#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cmath>
#include <numeric>

#include "../../include/louvain.h"
#include "exact.cuh"
#include "internal.h"
#include "mlp.cuh"

using namespace lv;
typedef __int128 i128;

namespace lv {
thread_local long long g_launches = 0;
}

struct PassTiming {
  cudaEvent_t t0, t1, t2;  // pass start, after local moving, after aggregation
  bool timed;              // t0 and t1 were recorded (false for passes restored from a checkpoint)
  bool aggregated;
};

// Where a run stands between two passes: what louvain_run_passes leaves for
// louvain_resume, and what a checkpoint holds besides the per-vertex arrays.
struct RunState {
  GView g{};          // current (super-)vertex graph
  int wk = 0;         // its weight kind
  int slot = 0;       // ping-pong buffer the next aggregation writes
  int next_pass = 0;  // index of the next pass (= passes completed)
  int64_t nnzp = 0;   // entries of g
  double tau = 0;     // tolerance of the next pass
};

struct louvain_ctx {
  louvain_config cfg;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  std::string err;

  int64_t n0 = 0, nnz0 = 0;
  long long two_m = 0;
  int weighted = 0;
  const int64_t *off0 = nullptr;
  const int32_t *col0 = nullptr;
  const int32_t *w0 = nullptr;

  // per-vertex state
  int32_t *C = nullptr, *Cp = nullptr;
  int64_t *K = nullptr, *Kalt = nullptr, *Sigma = nullptr;
  uint8_t *flag = nullptr;
  uint8_t *vbin = nullptr;  // move bin per vertex of the current pass
  uint32_t *recv = nullptr; // bit c: some vertex moved into community c this pass (known singletons)
  unsigned long long *wide_spill = nullptr;  // [SMs][kWideSpill] global tables of the wide bin (kept empty)
  bool rows_unique = false; // the input's rows are strictly increasing (no repeated column)
  // local moving
  int32_t *bins[kMoveBins] = {};
  int32_t *mv_vertex = nullptr, *mv_target = nullptr;
  // aggregation
  unsigned long long *cnt = nullptr, *cdeg = nullptr;
  int64_t *newid = nullptr, *coff = nullptr, *hoff = nullptr, *kcoff = nullptr;
  int32_t *members = nullptr, *kcnt = nullptr;
  long long *scan_tmp = nullptr;
  // ping-pong super-vertex graphs
  int32_t *pcol[2] = {};
  uint32_t *pw[2] = {};
  int64_t *pbeg[2] = {}, *pend[2] = {};
  // global tables of big items (hubs, large communities)
  BigWs big;
  bool big_dirty = false;
  // learned predictor and trace recorder
  float *mlp = nullptr;
  float4 *feat = nullptr;
  uint32_t *seen = nullptr;       // learned features: bucket stamps of evaluations and moves,
  uint32_t *moved_at = nullptr;   //   neighbour samples (see LearnArgs)
  int32_t *sample = nullptr;
  uint32_t *sample_n = nullptr;
  int32_t *sample_at = nullptr;
  int64_t sample_cap = 0;
  int2 *chunks = nullptr;
  int64_t chunk_cap = 0;
  uint32_t stamp = 0;             // stamp of the last bucket enqueued in the current pass
  // Leiden form (refine): refined partition and totals, per-vertex
  // refinement state, chunk records of long rows, and the next pass's
  // starting partition (linit) with its representatives (lrep)
  int32_t *Cr = nullptr;
  int64_t *Sr = nullptr;
  uint8_t *relig = nullptr, *rchosen = nullptr;
  unsigned long long *rkin = nullptr;
  int2 *rchunks = nullptr;
  int64_t rchunk_cap = 0;
  int32_t *linit = nullptr, *lrep = nullptr;
  int32_t *cand = nullptr;
  int32_t *skip_list = nullptr;  // learned: vertices skipped in the current iteration
  float *trace_x = nullptr, *trace_y = nullptr;
  int64_t trace_count = 0;
  std::vector<std::array<long long, 3>> learned_log;  // per pass: learned iterations, fallback iterations, last moves

  Counters *d_ctr = nullptr;
  Counters *h_ctr = nullptr;  // pinned

  std::vector<void *> allocs;
  size_t bytes = 0;

  // results of the last run
  bool ran = false;
  bool suspended = false;  // a run stopped between two passes (louvain_run_passes, louvain_load_state)
  RunState rs;
  uint64_t model_hash = 0; // of the learned predictor's parameters (checkpoint compatibility)
  double q = 0;
  i128 qnum = 0, qden = 0;
  int64_t gamma = 0;
  int passes = 0, exit_reason = 0;
  std::vector<int64_t> iter_stats, pass_stats;
  std::vector<PassTiming> timing;
  // iteration starts of every pass (iter_ev[p * (max_iterations + 1) + t]),
  // and the end of its local-moving phase at t = l_i; created on first use
  std::vector<cudaEvent_t> iter_ev;
  std::vector<int> iter_timed;  // per pass: iterations timed one by one (0: the phase as a whole)
  cudaEvent_t run0 = nullptr, run1 = nullptr;
  double run_ms = 0;
  long long it_total = 0, moves_total = 0, evaluated_total = 0, skipped_total = 0;
  long long launches = 0;
  // per-kernel profile of the last run
  KernelProf prof;
  std::vector<cudaEvent_t> prof_events;
  double kbytes[K_NUM_KERNELS] = {};
  double kunits[K_NUM_KERNELS][2] = {};  // work per kernel group: vertices (or communities), entries
  int cur_wbytes = 0;
  bool pass_has_hubs = false;
  int64_t hub_window = 0;
  int64_t hub_rounds = 0;
  long long *h_rounds = nullptr;     // pinned: rounds the current big items need
  cudaEvent_t plan_done = nullptr;
  Sched sched;                       // launch schedule (louvain_set_schedule / louvain_autotune)
  SideStreams side;                  // side streams for concurrent bin kernels
  // graph replay of local-moving iterations (sched.graphs)
  cudaGraphExec_t gexec = nullptr;
  long long graph_launches = 0;      // kernels per replay
  int graph_pass = -1;               // pass the executable graph was captured for
  bool graph_broken = false;         // a capture failed: direct launches for the rest of the run
  uint32_t *d_iter = nullptr;        // {salt, pickless} read by the kernels under replay
  uint32_t *h_iter = nullptr;        // pinned
  // device-controlled local-moving phase (sched.graphs = 2): one graph per
  // pass whose conditional while node repeats the iteration until the
  // device-side tolerance test ends it
  cudaGraphExec_t pexec = nullptr;
  int pexec_pass = -1;               // pass the phase graph was captured for
  bool phase_broken = false;         // a capture failed: host control for the rest of the run
  long long phase_launches = 0;      // kernels per iteration of the phase graph
  int32_t *d_phase = nullptr;        // {current iteration, iterations performed}
  unsigned long long *d_rec = nullptr;  // [max_iterations][kIterCounterWords] per-iteration counters
  int32_t *h_phase = nullptr;        // pinned copies
  unsigned long long *h_rec = nullptr;

  // batched runs: G graphs as one union graph (batch.cu)
  bool batched = false;
  int64_t G = 0;
  std::vector<int64_t> vo0;             // [G+1] vertex offsets of the input union
  std::vector<long long> gtwo_m;        // [G] 2m of each graph
  BatchView bview;                      // device view (gid == nullptr for a single graph)
  int32_t *b_gid = nullptr, *b_ogid = nullptr, *b_out = nullptr;
  int64_t *b_vo = nullptr, *b_bound = nullptr;
  long long *b_two_m = nullptr;
  int32_t *b_li = nullptr;              // [G] iterations of each graph's moving phase (device-controlled phase)
  int32_t *h_li = nullptr;              // pinned copy
  int8_t *b_moving = nullptr, *b_sel = nullptr;
  unsigned long long *b_acc = nullptr;  // [6][G]: gain lo, gain hi, moves, S_in, Sigma^2 lo, Sigma^2 hi
  unsigned long long *h_acc = nullptr;  // pinned copies
  int64_t *h_bound = nullptr;
  int8_t *h_flags = nullptr;
  std::vector<int64_t> b_results;       // [G][8]: passes, communities, Q num (hi, lo), Q den (hi, lo), 2m, exit
  std::vector<double> b_q;              // [G]
  std::vector<int64_t> b_passes;        // [G][max_passes][3]: n', l_i, |Gamma|
  std::vector<void *> pinned;           // pinned host buffers (freed by destroy)
};

namespace {

thread_local std::string g_create_err;

#define LV_CK(call)                                                                         \
  do {                                                                                      \
    cudaError_t e__ = (call);                                                               \
    if (e__ != cudaSuccess) {                                                               \
      set_err(x, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e__), __FILE__, __LINE__); \
      return LOUVAIN_E_CUDA;                                                                \
    }                                                                                       \
  } while (0)

void set_err(louvain_ctx *x, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (x) x->err = buf;
  else g_create_err = buf;
}

louvain_status dalloc(louvain_ctx *x, void **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, x->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_err(x, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return LOUVAIN_E_NOMEM;
  }
  x->allocs.push_back(*p);
  x->bytes += bytes;
  return LOUVAIN_OK;
}

template <class T>
louvain_status dalloc_n(louvain_ctx *x, T **p, int64_t n) {
  return dalloc(x, (void **)p, (size_t)(n > 0 ? n : 1) * sizeof(T));
}

void release_pool_threshold(int device) {
  static bool done[64] = {};
  if (device < 0 || device >= 64 || done[device]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[device] = true;
}

// Input validation: offsets non-decreasing (thread per row), then every
// entry's column in [0, n) and weight > 0, with the weights summed into 2m
// (thread per entry, coalesced); per-warp reductions before the atomics.
// Both kernels also count descents, adjacent entries with col[k-1] >=
// col[k]: all of them (entries) and those where k starts a non-empty row
// (rows).  Every row is strictly increasing, so holds no repeated column,
// exactly when the two counts agree (descents[0] == descents[1]).
__global__ void k_validate_rows(int64_t n, const int64_t *off, const int32_t *col, Counters *ctr) {
  bool bad = false;
  unsigned long long starts = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = off[i], e = off[i + 1];
    if (e < b) bad = true;
    else if (b > 0 && e > b && col[b - 1] >= col[b]) ++starts;  // b - 1 ends the previous non-empty row
  }
  starts = warp_sum_u(starts);
  if ((threadIdx.x & 31) == 0 && starts) atomicAdd(&ctr->descents[1], starts);
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(&ctr->error, (unsigned long long)ERR_RANGE);
}

// Entries of a CSR (input int32 weights, or the uint32 weights of a
// super-vertex graph restored from a checkpoint): column in [0, n), weight
// > 0; the weights are summed into ctr->q_sin.
template <typename WT>
__global__ void k_validate_entries(int64_t nnz, int64_t n, const int32_t *col, const WT *w, Counters *ctr) {
  bool bad = false;
  unsigned long long wsum = 0, desc = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = col[k];
    if (c < 0 || c >= n) bad = true;
    if (k > 0 && col[k - 1] >= c) ++desc;
    const WT ww = w ? w[k] : WT(1);
    if (ww <= WT(0)) bad = true;
    wsum += (unsigned long long)(ww > WT(0) ? ww : WT(0));
  }
  wsum = warp_sum_u(wsum);
  desc = warp_sum_u(desc);
  const bool any_bad = __any_sync(0xFFFFFFFFu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (any_bad) atomicOr(&ctr->error, (unsigned long long)ERR_RANGE);
    if (wsum) atomicAdd(&ctr->q_sin, wsum);
    if (desc) atomicAdd(&ctr->descents[0], desc);
  }
}

// End of one local-moving iteration when the whole phase runs under device
// control (a conditional while node): the iteration's counters are kept in
// rec[t], the tolerance test of Algorithm 2 is taken with the host's exact
// arithmetic (the 128-bit gain, correctly rounded conversions, one double
// division), and either the next iteration's salt and Pick-Less flag are
// set or the loop ends (phase[1] = iterations performed).
struct PhaseStep {
  long long two_m;
  double tau;
  int max_it, pass, rho;
  uint64_t seed;
};
__global__ void k_phase_step(const Counters *ctr, uint32_t *iter, int32_t *phase, unsigned long long *rec, PhaseStep p,
                             cudaGraphConditionalHandle handle) {
  const int t = phase[0];
  const unsigned long long *w = &ctr->it_gain_lo;
  for (int k = threadIdx.x; k < kIterCounterWords; k += blockDim.x) rec[(size_t)t * kIterCounterWords + k] = w[k];
  if (threadIdx.x != 0) return;
  const unsigned long long glo = ctr->it_gain_lo, ghi = ctr->it_gain_hi;
  const unsigned long long lo = glo + (ghi << 32);                 // gain = ghi 2^32 + glo
  const unsigned long long hi = (ghi >> 32) + (lo < glo ? 1ull : 0ull);
  const unsigned long long tlo = lo << 1, thi = (hi << 1) | (lo >> 63);  // 2 gain
  const unsigned long long den2 = (unsigned long long)p.two_m * (unsigned long long)p.two_m;  // (2m)^2 < 2^64
  const double total = den2 ? u128_to_double(thi, tlo) / u128_to_double(0, den2) : 0.0;
  const bool stop = total <= p.tau || t + 1 >= p.max_it;
  if (stop) {
    phase[1] = t + 1;
  } else {
    phase[0] = t + 1;
    iter[0] = bucket_salt(p.pass, t + 1, p.seed);
    iter[1] = (p.rho > 0 && ((t + 1 + p.rho / 2) % p.rho) == 0) ? 1u : 0u;
  }
  cudaGraphSetConditional(handle, stop ? 0u : 1u);
}

// The same for a batch: every graph still moving takes its own tolerance
// test with its own 2m (its gain sums in gain_lo/gain_hi); a graph that
// meets it stops moving (moving[k] = 0, li[k] = t + 1).  The loop ends when
// no graph moves or at the iteration cap.  One block.
__global__ void __launch_bounds__(1024) k_batch_phase_step(const Counters *ctr, uint32_t *iter, int32_t *phase,
                                                           unsigned long long *rec, PhaseStep p,
                                                           const unsigned long long *gain_lo,
                                                           const unsigned long long *gain_hi,
                                                           const long long *two_m, int8_t *moving, int32_t *li,
                                                           int64_t G, cudaGraphConditionalHandle handle) {
  const int t = phase[0];
  const unsigned long long *w = &ctr->it_gain_lo;
  for (int k = threadIdx.x; k < kIterCounterWords; k += blockDim.x) rec[(size_t)t * kIterCounterWords + k] = w[k];
  bool any = false;
  for (int64_t k = threadIdx.x; k < G; k += blockDim.x) {
    if (!moving[k]) continue;
    const unsigned long long glo = gain_lo[k], ghi = gain_hi[k];
    const unsigned long long lo = glo + (ghi << 32);
    const unsigned long long hi = (ghi >> 32) + (lo < glo ? 1ull : 0ull);
    const unsigned long long den2 = (unsigned long long)two_m[k] * (unsigned long long)two_m[k];
    const double total = den2 ? u128_to_double((hi << 1) | (lo >> 63), lo << 1) / u128_to_double(0, den2) : 0.0;
    if (total <= p.tau) {
      moving[k] = 0;
      li[k] = t + 1;
    } else {
      any = true;
    }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x != 0) return;
  const bool stop = !any || t + 1 >= p.max_it;
  if (stop) {
    phase[1] = t + 1;
  } else {
    phase[0] = t + 1;
    iter[0] = bucket_salt(p.pass, t + 1, p.seed);
    iter[1] = (p.rho > 0 && ((t + 1 + p.rho / 2) % p.rho) == 0) ? 1u : 0u;
  }
  cudaGraphSetConditional(handle, stop ? 0u : 1u);
}

// Rows of a holey CSR copied to consecutive positions (row i to off[i]),
// one warp per row.
__global__ void k_compact_rows(int64_t n, const int64_t *b, const int64_t *e, const int64_t *off, const int32_t *cs,
                               const uint32_t *ws, int32_t *cd, uint32_t *wd) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    const int64_t b0 = b[i], len = e[i] - b0, o = off[i];
    for (int64_t k = lane; k < len; k += 32) {
      cd[o + k] = cs[b0 + k];
      wd[o + k] = ws[b0 + k];
    }
  }
}

void dfree(louvain_ctx *x, void *p) {
  if (!p) return;
  cudaFreeAsync(p, x->stream);
  auto it = std::find(x->allocs.begin(), x->allocs.end(), p);
  if (it != x->allocs.end()) x->allocs.erase(it);
}

// Grow the big-item workspace to `slots` table slots, `parts` evaluation
// partials and `items` items; new tables are cleared (all keys empty).
louvain_status ensure_big(louvain_ctx *x, int64_t slots, int64_t parts, int64_t items, int64_t rounds) {
  louvain_status st;
  BigWs &b = x->big;
  if (!b.nrounds) {
    if ((st = dalloc_n(x, &b.nrounds, 1))) return st;
    if (cudaMallocHost((void **)&x->h_rounds, sizeof(long long)) != cudaSuccess) {
      set_err(x, "pinned allocation failed");
      return LOUVAIN_E_NOMEM;
    }
    LV_CK(cudaEventCreateWithFlags(&x->plan_done, cudaEventDisableTiming));
  }
  if (rounds > b.round_cap) {
    dfree(x, b.rstart);
    b.rstart = nullptr;
    const int64_t want = rounds + rounds / 4 + 8;
    if ((st = dalloc_n(x, &b.rstart, want + 2))) return st;
    b.round_cap = want;
  }
  if (slots > b.slots) {
    dfree(x, b.tab);
    dfree(x, b.occ);
    b.tab = nullptr;
    b.occ = nullptr;
    b.slots = 0;
    const int64_t want = slots + slots / 4;
    if ((st = dalloc_n(x, &b.tab, want)) || (st = dalloc_n(x, &b.occ, want / 2 + 1))) return st;
    LV_CK(cudaMemsetAsync(b.tab, 0, (size_t)want * sizeof(unsigned long long), x->stream));
    b.slots = want;
  }
  if (parts > b.parts) {
    dfree(x, b.part_s);
    dfree(x, b.part_c);
    dfree(x, b.part_kid);
    const int64_t want = parts + parts / 4 + 64;
    if ((st = dalloc_n(x, &b.part_s, want)) || (st = dalloc_n(x, &b.part_c, want)) ||
        (st = dalloc_n(x, &b.part_kid, want)))
      return st;
    b.parts = want;
  }
  if (items > b.item_cap) {
    dfree(x, b.tot);
    dfree(x, b.toff);
    dfree(x, b.cpre);
    dfree(x, b.epre);
    dfree(x, b.ocnt);
    const int64_t want = items + items / 4 + 64;
    if ((st = dalloc_n(x, &b.tot, want + 1)) || (st = dalloc_n(x, &b.toff, want + 1)) ||
        (st = dalloc_n(x, &b.cpre, want + 1)) || (st = dalloc_n(x, &b.epre, want + 1)) ||
        (st = dalloc_n(x, &b.ocnt, want + 1)))
      return st;
    b.item_cap = want;
  }
  return LOUVAIN_OK;
}

// Workspace for the big items counted in ctr->big_slots / big_items (their
// tables' total size, a bound for every bucket), largest item `maxdeg` over
// `keyspace` keys: tables go through a window of about half the total per
// round (a bucket holds about 1/B of the pass's items, so one or two rounds
// run), the workspace is window + the largest table, and rstart holds the
// rounds of the total.
louvain_status ensure_big_for(louvain_ctx *x, const Counters &h, uint64_t maxdeg, uint64_t keyspace, int64_t *window,
                              int64_t *rounds) {
  *window = 0;
  *rounds = 0;
  if (h.big_items == 0) return LOUVAIN_OK;
  const int64_t total = (int64_t)h.big_slots;
  const int64_t maxcap = (int64_t)big_table_cap(maxdeg, keyspace);
  const int64_t target = x->cfg.table_window > 0 ? x->cfg.table_window : (total + 1) / 2;
  int64_t w = ((std::min<int64_t>(total, target)) + 63) & ~63ll;
  if (w < maxcap) w = maxcap;
  int64_t r = (total + w - 1) / w;
  if (r < 1) r = 1;
  *window = w;
  *rounds = r;
  return ensure_big(x, w + maxcap, total / kBigEvalSlots + (int64_t)h.big_items + 1, (int64_t)h.big_items + 1, r);
}

louvain_status read_counters(louvain_ctx *x) {
  LV_CK(cudaMemcpyAsync(x->h_ctr, x->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, x->stream));
  LV_CK(cudaStreamSynchronize(x->stream));
  if (x->h_ctr->error & ERR_HASH) {
    set_err(x, "a hashtable insert exceeded its probe limit (the failed result of Algorithm 7)");
    return LOUVAIN_E_HASH_OVERFLOW;
  }
  return LOUVAIN_OK;
}

// FNV-1a (Fowler, Noll, Vo), 64-bit, over bytes: fingerprints of
// checkpoint payloads, configurations and model parameters.
uint64_t fnv1a_bytes(const void *p, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

void put128(int64_t *dst, i128 v) {
  dst[0] = (int64_t)(v >> 64);
  dst[1] = (int64_t)(uint64_t)v;
}

// Algorithmic bytes of one iteration's kernels (what the method must move):
// decide, per vertex: bin entry 4, row bounds 16, C'[i] 4, K_i 8, Sigma_d 8;
// per entry: column 4 + weight + C'[j] 4; per distinct candidate: Sigma_c 8;
// per mover: decision 8 + one flag byte per neighbour.  select: one flag byte
// per vertex per bucket, plus flag write, row bounds and list entry of the
// selected.  apply: decision 8, C' read/write 8, K_i 8, two Sigma atomics 16.
void account_move(louvain_ctx *x, int64_t n, const Counters &h) {
  if (x->prof.mask) x->prof.collect();
  const double wb = x->cur_wbytes;
  for (int b = 0; b < kMoveBins; ++b) {
    const unsigned long long *w = h.mv_work[b];
    if (b == kBigBin) {  // entries in the accumulation kernel, the rest in evaluation
      x->kbytes[K_MOVE_HUB] += (8.0 + wb) * w[1];
      x->kbytes[K_MOVE_HUB_EVAL] += 40.0 * w[0] + 8.0 * w[2] + 8.0 * w[3] + 1.0 * w[4];
      x->kunits[K_MOVE_HUB][0] += (double)w[0];
      x->kunits[K_MOVE_HUB][1] += (double)w[1];
      continue;
    }
    const int kid = b == kGroupBin     ? K_MOVE_GROUP
                    : b == kXlBin      ? K_MOVE_XL
                    : b == kHalfBin    ? K_MOVE_HALF
                                       : K_MOVE_THREAD + b;
    x->kbytes[kid] += 40.0 * w[0] + (8.0 + wb) * w[1] + 8.0 * w[2] + 8.0 * w[3] + 1.0 * w[4];
    x->kunits[kid][0] += (double)w[0];
    x->kunits[kid][1] += (double)w[1];
  }
  const int nbuckets = x->cfg.asynchronous ? 1 : x->cfg.buckets;
  x->kbytes[K_SELECT] += (double)nbuckets * n + 21.0 * h.it_evaluated;
  if (!x->cfg.asynchronous) x->kbytes[K_APPLY] += 40.0 * h.it_moves;  // the asynchronous form applies in place
}

// Aggregation kernels: per community: member offset/count 12, row bounds 16,
// row end write 8; per member: id 4, row bounds 16; per entry: column 4 +
// weight + C'[j] 4; per output entry: 8 (id and uint32 weight).
void account_merge(louvain_ctx *x, const Counters &h) {
  if (x->prof.mask) x->prof.collect();
  const double wb = x->cur_wbytes;
  for (int b = 0; b < kMergeBins; ++b) {
    const unsigned long long *w = h.mg_work[b];
    if (b == kBigBin) {
      x->kbytes[K_MERGE_BIG] += 20.0 * w[1] + (8.0 + wb) * w[2];
      x->kbytes[K_MERGE_BIG_EMIT] += 36.0 * w[0] + 8.0 * w[3];
      x->kunits[K_MERGE_BIG][0] += (double)w[0];
      x->kunits[K_MERGE_BIG][1] += (double)w[2];
      continue;
    }
    const int kid = b == kMergeXlBin ? K_MERGE_XL : b == kMergeGroupBin ? K_MERGE_GROUP : K_MERGE_THREAD + b;
    x->kbytes[kid] += 36.0 * w[0] + 20.0 * w[1] + (8.0 + wb) * w[2] + 8.0 * w[3];
    x->kunits[kid][0] += (double)w[0];
    x->kunits[kid][1] += (double)w[2];
  }
}

LearnArgs learn_args(louvain_ctx *x, int pass, int t, bool skipping) {
  const louvain_config &cfg = x->cfg;
  LearnArgs L;
  L.record = x->feat != nullptr;
  L.enabled = skipping && cfg.mode == LOUVAIN_MODE_LEARNED;
  L.params = x->mlp;
  L.feat = x->feat;
  L.seen = x->seen;
  L.moved_at = L.record ? x->moved_at : nullptr;
  L.sample = x->sample;
  L.sample_n = x->sample_n;
  L.sample_at = x->sample_at;
  L.sample_cap = x->sample_cap;
  L.chunks = x->chunks;
  L.chunk_cap = x->chunk_cap;
  L.stamp = x->stamp;
  L.cand = x->cand;
  const double th = std::min(std::max((double)cfg.skip_threshold, 1e-6), 1.0 - 1e-6);
  L.thr_logit = (float)std::log(th / (1.0 - th));
  L.skip_clears = cfg.learned_skip_clears;
  L.min_degree = cfg.learned_min_degree;
  L.vbin = x->vbin;
  if (cfg.learned_fallback == 3) L.skip_list = x->skip_list;
  L.t_norm = (float)t / (float)cfg.max_iterations;
  L.p_norm = (float)pass / (float)std::max(cfg.max_passes, 1);
  if (x->trace_x) {
    L.trace_x = x->trace_x;
    L.trace_y = x->trace_y;
    L.trace_cap = cfg.trace_capacity;
    const double r = std::min(std::max((double)cfg.trace_rate, 0.0), 1.0);
    L.trace_keep = (uint32_t)std::lround(r * 65536.0);
    L.trace_salt = fmix32(0x7261ce5u ^ ((uint32_t)pass << 8) ^ (uint32_t)t);
  }
  return L;
}

// One iteration of the local-moving phase (all buckets); fills *h.  With
// `completion`, the completion step of learned iteration t instead: the
// vertices the predictor skipped in it are evaluated, and the counts and gain
// are added to iteration t's record.
louvain_status move_iteration(louvain_ctx *x, const GView &g, int wk, int pass, int t, bool skipping,
                              const Counters **h_out, bool completion = false);
louvain_status begin_run(louvain_ctx *x);

louvain_status enqueue_iteration(louvain_ctx *x, const GView &g, int wk, int pass, int t, bool skipping,
                                 const uint32_t *iter, bool completion);
void record_iteration(louvain_ctx *x, const GView &g, int pass, int t, const Counters &h, bool completion);
louvain_status mark_iteration(louvain_ctx *x, int pass, int t);

// The phase graph of a pass: a conditional while node whose body is one
// local-moving iteration (the kernels read the salt and Pick-Less flag from
// x->d_iter) followed by k_phase_step, which ends the loop on the device.
// A capture that fails sets phase_broken (host control from then on).
louvain_status capture_phase(louvain_ctx *x, const GView &g, int wk, int pass, double tau) {
  const louvain_config &cfg = x->cfg;
  cudaStream_t s = x->stream;
  louvain_status st;
  if (!x->d_iter) {
    if ((st = dalloc_n(x, &x->d_iter, 2))) return st;
    if (cudaMallocHost((void **)&x->h_iter, 2 * sizeof(uint32_t)) != cudaSuccess) {
      set_err(x, "pinned allocation failed");
      return LOUVAIN_E_NOMEM;
    }
  }
  if (!x->d_phase) {
    const size_t words = (size_t)cfg.max_iterations * kIterCounterWords;
    if ((st = dalloc_n(x, &x->d_phase, 2)) || (st = dalloc_n(x, &x->d_rec, (int64_t)words))) return st;
    if (cudaMallocHost((void **)&x->h_phase, 2 * sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost((void **)&x->h_rec, words * sizeof(unsigned long long)) != cudaSuccess) {
      set_err(x, "pinned allocation failed");
      return LOUVAIN_E_NOMEM;
    }
  }
  if (x->pexec) {
    cudaGraphExecDestroy(x->pexec);
    x->pexec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphConditionalHandle handle;
  cudaGraphNodeParams cp{};
  cudaGraphNode_t node;
  bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
  }
  const long long l0 = g_launches;
  if (ok) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      st = enqueue_iteration(x, g, wk, pass, 0, false, x->d_iter, false);
      const PhaseStep ps{x->two_m, tau, cfg.max_iterations, pass, cfg.pickless_period, cfg.schedule_seed};
      if (x->batched)
        LV_LAUNCH(k_batch_phase_step<<<1, 1024, 0, s>>>(x->d_ctr, x->d_iter, x->d_phase, x->d_rec, ps,
                                                         x->bview.gain_lo, x->bview.gain_hi, x->b_two_m, x->b_moving,
                                                         x->b_li, x->G, handle));
      else
        LV_LAUNCH(k_phase_step<<<1, 64, 0, s>>>(x->d_ctr, x->d_iter, x->d_phase, x->d_rec, ps, handle));
      cudaGraph_t captured = nullptr;
      ok = cudaStreamEndCapture(s, &captured) == cudaSuccess && st == LOUVAIN_OK;
    }
  }
  x->phase_launches = g_launches - l0;
  g_launches = l0;
  if (ok) ok = cudaGraphInstantiate(&x->pexec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();
    if (x->pexec) cudaGraphExecDestroy(x->pexec);
    x->pexec = nullptr;
    x->phase_broken = true;
    return LOUVAIN_OK;
  }
  x->pexec_pass = pass;
  return LOUVAIN_OK;
}

// The local-moving phase of a plain pass under device control: one graph
// launch, one synchronisation, then the per-iteration records (for a batch
// also each graph's iteration count, in x->h_li; the caller has set every
// graph's moving flag and b_li = max_iterations).
louvain_status device_phase(louvain_ctx *x, const GView &g, int wk, int pass, double tau, int *li_out) {
  const louvain_config &cfg = x->cfg;
  louvain_status st;
  if (x->pexec_pass != pass && (st = capture_phase(x, g, wk, pass, tau))) return st;
  if (x->phase_broken) return LOUVAIN_OK;
  const int rho = cfg.pickless_period;
  x->h_iter[0] = bucket_salt(pass, 0, cfg.schedule_seed);
  x->h_iter[1] = (rho > 0 && ((0 + rho / 2) % rho) == 0) ? 1u : 0u;
  LV_CK(cudaMemcpyAsync(x->d_iter, x->h_iter, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice, x->stream));
  LV_CK(cudaMemsetAsync(x->d_phase, 0, 2 * sizeof(int32_t), x->stream));
  if ((size_t)pass < x->iter_timed.size()) x->iter_timed[pass] = 0;  // timed as a whole
  if ((st = mark_iteration(x, pass, 0))) return st;
  LV_CK(cudaGraphLaunch(x->pexec, x->stream));
  LV_CK(cudaMemcpyAsync(x->h_phase, x->d_phase, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, x->stream));
  LV_CK(cudaMemcpyAsync(x->h_rec, x->d_rec, (size_t)cfg.max_iterations * kIterCounterWords * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, x->stream));
  if (x->batched)
    LV_CK(cudaMemcpyAsync(x->h_li, x->b_li, (size_t)x->G * sizeof(int32_t), cudaMemcpyDeviceToHost, x->stream));
  if ((st = read_counters(x))) return st;  // synchronises; hashtable errors of any iteration
  const int li = x->h_phase[1];
  if (li < 1 || li > cfg.max_iterations) {
    set_err(x, "device-controlled local moving ended after %d iterations", li);
    return LOUVAIN_E_CUDA;
  }
  g_launches += x->phase_launches * li;
  for (int t = 0; t < li; ++t) {
    Counters h{};
    memcpy(&h.it_gain_lo, x->h_rec + (size_t)t * kIterCounterWords, kIterCounterWords * sizeof(unsigned long long));
    record_iteration(x, g, pass, t, h, false);
  }
  *li_out = li;
  return LOUVAIN_OK;
}

// Event at iteration t of pass p (t = l_i: the end of the phase).
louvain_status mark_iteration(louvain_ctx *x, int pass, int t) {
  const size_t k = (size_t)pass * (x->cfg.max_iterations + 1) + t;
  if (k >= x->iter_ev.size()) return LOUVAIN_OK;
  if (!x->iter_ev[k]) LV_CK(cudaEventCreate(&x->iter_ev[k]));
  LV_CK(cudaEventRecord(x->iter_ev[k], x->stream));
  return LOUVAIN_OK;
}

// Local-moving phase (Algorithm 5) under the bucket schedule; returns l_i.
// Plain single-graph runs with sched.graphs = 2 run it under device control
// (device_phase); the result is the same as the host-controlled loop's.
// Learned mode with completion (learned_fallback 3): iterations with the
// predictor; when an iteration's gain meets the tolerance, the vertices it
// skipped are evaluated at once (its completion step, gains added to the
// iteration's), and the phase ends only if the iteration's total still
// meets it: the plain stopping rule, checked on every vertex the iteration
// would have evaluated without the predictor.  Learned mode otherwise:
// iterations with the predictor until the tolerance is met, then plain
// iterations (learned_fallback 0, 1, 2).
louvain_status move_phase_impl(louvain_ctx *x, const GView &g, int wk, int pass, double tau, int *li_out) {
  const louvain_config &cfg = x->cfg;
  if (cfg.mode == LOUVAIN_MODE_LEARNED && cfg.learned_fallback == 3) {
    const i128 den2 = (i128)x->two_m * x->two_m;
    int li = cfg.max_iterations;
    long long completions = 0, last_moves = -1;
    for (int t = 0; t < cfg.max_iterations; ++t) {
      const Counters *h;
      louvain_status st = move_iteration(x, g, wk, pass, t, true, &h);
      if (st) return st;
      i128 gain = ((i128)h->it_gain_hi << 32) + (i128)h->it_gain_lo;
      last_moves = (long long)h->it_moves;
      double total = den2 ? (double)(2 * gain) / (double)den2 : 0.0;
      if (total > tau) continue;
      if (h->skip_listed > 0) {  // the completion step judges the iteration
        const Counters *hc;
        if ((st = move_iteration(x, g, wk, pass, t, false, &hc, true))) return st;
        ++completions;
        last_moves += (long long)hc->it_moves;
        gain += ((i128)hc->it_gain_hi << 32) + (i128)hc->it_gain_lo;
        total = den2 ? (double)(2 * gain) / (double)den2 : 0.0;
      }
      if (total <= tau) {
        li = t + 1;
        break;
      }
    }
    x->learned_log.push_back({(long long)li, completions, last_moves});
    *li_out = li;
    return LOUVAIN_OK;
  }
  if (cfg.mode == LOUVAIN_MODE_LEARNED) {
    const i128 den2 = (i128)x->two_m * x->two_m;
    int t = 0;
    for (; t < cfg.max_iterations; ++t) {
      const Counters *h;
      louvain_status st = move_iteration(x, g, wk, pass, t, true, &h);
      if (st) return st;
      const i128 gain = ((i128)h->it_gain_hi << 32) + (i128)h->it_gain_lo;
      const double total = den2 ? (double)(2 * gain) / (double)den2 : 0.0;
      if (total <= tau) {
        ++t;
        break;
      }
    }
    // fallback: plain iterations without the predictor over the flagged
    // vertices (every skipped vertex kept its flag) or, on request, over all
    // vertices first; until the plain tolerance test holds or, on request,
    // until an iteration makes no move
    const int learned_iters = t;
    long long last_moves = -1;
    if (cfg.learned_fallback != 0) flag_all(x->flag, g.n, x->num_sms, x->stream);
    for (int f = 0; f < cfg.max_iterations; ++f, ++t) {
      const Counters *h;
      louvain_status st = move_iteration(x, g, wk, pass, t, false, &h);
      if (st) return st;
      last_moves = (long long)h->it_moves;
      const i128 gain = ((i128)h->it_gain_hi << 32) + (i128)h->it_gain_lo;
      const double total = den2 ? (double)(2 * gain) / (double)den2 : 0.0;
      if (cfg.learned_fallback == 1 ? h->it_moves == 0 : total <= tau) {
        ++t;
        break;
      }
    }
    x->learned_log.push_back({(long long)learned_iters, (long long)(t - learned_iters), last_moves});
    *li_out = t;
    return LOUVAIN_OK;
  }
  if (x->sched.graphs == 2 && !x->batched && !x->prof.mask && !x->trace_x && !x->phase_broken &&
      cfg.mode == LOUVAIN_MODE_PLAIN) {
    louvain_status st = device_phase(x, g, wk, pass, tau, li_out);
    if (st || !x->phase_broken) return st;
  }
  const i128 den2 = (i128)x->two_m * x->two_m;
  int li = cfg.max_iterations;
  for (int t = 0; t < cfg.max_iterations; ++t) {
    const Counters *hp;
    louvain_status st = move_iteration(x, g, wk, pass, t, false, &hp);
    if (st) return st;
    const Counters &h = *hp;
    const i128 gain = ((i128)h.it_gain_hi << 32) + (i128)h.it_gain_lo;
    const double total = den2 ? (double)(2 * gain) / (double)den2 : 0.0;
    if (total <= tau) {
      li = t + 1;
      break;
    }
  }
  *li_out = li;
  return LOUVAIN_OK;
}

louvain_status move_phase(louvain_ctx *x, const GView &g, int wk, int pass, double tau, int *li_out) {
  if ((size_t)pass < x->iter_timed.size()) x->iter_timed[pass] = 1;
  louvain_status st = move_phase_impl(x, g, wk, pass, tau, li_out);
  if (st) return st;
  return mark_iteration(x, pass, *li_out);
}

// Bookkeeping of one iteration from its counters: bytes per kernel, the
// per-iteration record (added to iteration t's with `completion`), totals.
void record_iteration(louvain_ctx *x, const GView &g, int pass, int t, const Counters &h, bool completion) {
  const louvain_config &cfg = x->cfg;
  const i128 gain = ((i128)h.it_gain_hi << 32) + (i128)h.it_gain_lo;
  account_move(x, g.n, h);
  if (pass < cfg.max_passes && t < cfg.max_iterations) {
    int64_t *r = &x->iter_stats[((size_t)pass * cfg.max_iterations + t) * 4];
    i128 g0 = 0;
    if (completion) g0 = ((i128)r[2] << 64) + (i128)(uint64_t)r[3];
    r[0] = (completion ? r[0] : 0) + (int64_t)h.it_evaluated;
    r[1] = (completion ? r[1] : 0) + (int64_t)h.it_moves;
    put128(r + 2, g0 + gain);
  }
  if (!completion) x->it_total += 1;
  x->moves_total += (long long)h.it_moves;
  x->evaluated_total += (long long)h.it_evaluated;
  x->skipped_total += (long long)h.it_skipped;
}

// Launches of one local-moving iteration (all buckets) on x->stream; with
// `iter` the kernels read the salt and Pick-Less flag from device memory and
// the hub path launches its rounds without asking (graph capture).
louvain_status enqueue_iteration(louvain_ctx *x, const GView &g, int wk, int pass, int t, bool skipping,
                                 const uint32_t *iter, bool completion) {
  const louvain_config &cfg = x->cfg;
  {
    const int rho = cfg.pickless_period;
    const LearnArgs L = learn_args(x, pass, t, skipping && t > 0 && !completion);
    const int pickless = rho > 0 && ((t + rho / 2) % rho) == 0;
    LV_CK(cudaMemsetAsync(&x->d_ctr->it_gain_lo, 0, kIterCounterWords * sizeof(unsigned long long), x->stream));
    if (L.enabled && L.skip_list)
      LV_CK(cudaMemsetAsync(&x->d_ctr->skip_listed, 0, sizeof(unsigned long long), x->stream));
    if (x->batched) LV_CK(cudaMemsetAsync(x->b_acc, 0, 3 * (size_t)x->G * sizeof(unsigned long long), x->stream));
    MoveArgs a{};
    a.g = g;
    a.Cp = x->Cp;
    a.K = x->K;
    a.Sigma = x->Sigma;
    a.flag = x->flag;
    a.two_m = x->two_m;
    a.pickless = pickless;
    a.salt = bucket_salt(pass, t, cfg.schedule_seed);
    const int nbuckets = cfg.asynchronous ? 1 : cfg.buckets;  // the asynchronous form sweeps all vertices at once
    a.nbuckets = (uint32_t)nbuckets;
    a.async_apply = cfg.asynchronous;
    for (int k = 0; k < kMoveBins; ++k) a.bins[k] = x->bins[k];
    a.mv_vertex = x->mv_vertex;
    a.mv_target = x->mv_target;
    a.ctr = x->d_ctr;
    a.learn = L;
    a.batch = x->bview;
    a.sched = x->sched;
    a.iter = iter;
    a.vbin = x->vbin;
    a.recv = x->recv;
    a.wide_spill = x->wide_spill;
    // known singletons need rows without repeated columns: super-vertex rows
    // have none, the input's were checked by louvain_create
    a.solo = !cfg.asynchronous && (pass > 0 || x->rows_unique);
    if (completion) {
      a.sel_list = x->skip_list;
      a.sel_count = &x->d_ctr->skip_listed;
    }
    BigArgs big{};
    big.g = g;
    big.Cp = x->Cp;
    big.items = x->bins[kBigBin];
    big.count = &x->d_ctr->bin_count[kBigBin];
    big.keyspace = g.n;
    big.ws = x->big;
    big.window = x->hub_window;
    big.rounds = x->hub_rounds;
    big.h_rounds = x->h_rounds;
    big.plan_done = x->plan_done;
    if (!x->pass_has_hubs) big.ws.slots = 0;
    big.ctr = x->d_ctr;
    big.K = x->K;
    big.Sigma = x->Sigma;
    big.flag = x->flag;
    big.two_m = x->two_m;
    big.pickless = pickless;
    big.mv_vertex = x->mv_vertex;
    big.mv_target = x->mv_target;
    big.async_apply = cfg.asynchronous;
    big.apply_Cp = x->Cp;
    big.apply_Sigma = x->Sigma;
    big.learn = L;
    big.batch = x->bview;
    big.accum_blocks = x->sched.move[kBigBin];
    big.iter = iter;
    big.static_rounds = iter != nullptr;
    for (int b = 0; b < (completion ? 1 : nbuckets); ++b) {
      LV_CK(cudaMemsetAsync(x->d_ctr, 0, offsetof(Counters, it_gain_lo), x->stream));
      if (L.enabled) LV_CK(cudaMemsetAsync(&x->d_ctr->cand_count, 0, sizeof(unsigned long long), x->stream));
      a.bucket = (uint32_t)b;
      if (L.record) a.learn.stamp = big.learn.stamp = ++x->stamp;  // every bucket (and completion step) a later stamp
      move_bucket(a, big, wk, x->num_sms, x->stream, x->prof.mask ? &x->prof : nullptr,
                  x->side.fork ? &x->side : nullptr);
    }
  }
  return LOUVAIN_OK;
}

// Capture the iteration's launches into x->gexec (once per pass).
louvain_status capture_iteration(louvain_ctx *x, const GView &g, int wk, int pass) {
  cudaStream_t s = x->stream;
  if (!x->d_iter) {
    louvain_status st;
    if ((st = dalloc_n(x, &x->d_iter, 2))) return st;
    if (cudaMallocHost((void **)&x->h_iter, 2 * sizeof(uint32_t)) != cudaSuccess) {
      set_err(x, "pinned allocation failed");
      return LOUVAIN_E_NOMEM;
    }
  }
  cudaGraph_t graph = nullptr;
  const long long l0 = g_launches;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    x->graph_broken = true;
    return LOUVAIN_OK;
  }
  louvain_status st = enqueue_iteration(x, g, wk, pass, 0, false, x->d_iter, false);
  const cudaError_t ec = cudaStreamEndCapture(s, &graph);
  x->graph_launches = g_launches - l0;
  g_launches = l0;
  if (st != LOUVAIN_OK || ec != cudaSuccess || !graph) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    x->graph_broken = true;
    return LOUVAIN_OK;
  }
  bool ok = false;
  if (x->gexec) {
    cudaGraphExecUpdateResultInfo info;
    ok = cudaGraphExecUpdate(x->gexec, graph, &info) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      cudaGraphExecDestroy(x->gexec);
      x->gexec = nullptr;
    }
  }
  if (!ok) ok = cudaGraphInstantiate(&x->gexec, graph, 0) == cudaSuccess;
  cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();
    x->gexec = nullptr;
    x->graph_broken = true;
    return LOUVAIN_OK;
  }
  x->graph_pass = pass;
  return LOUVAIN_OK;
}

// The refinement's sweep runs over this many buckets per bucket B of local
// moving (Leiden visits vertices one at a time, each seeing the merges made
// before it; more buckets make fewer decisions simultaneous).
constexpr int kRefineBucketsPerB = 4;

// Leiden refinement of P = C' on G' (the refine field of include/louvain.h):
// the filtered rows go to the ping-pong buffer that this pass's aggregation
// writes afterwards; one sweep over the 4B buckets of (vertex, pass,
// iteration 255) runs the local-moving decision kernels on the filtered view
// with the refined partition, and resolve + flags after every bucket.
louvain_status refine_phase(louvain_ctx *x, const GView &g, int wk, int slot, int pass) {
  const louvain_config &cfg = x->cfg;
  cudaStream_t s = x->stream;
  RefineArgs r{};
  r.g = g;
  r.Cp = x->Cp;
  r.K = x->K;
  r.Sigma = x->Sigma;
  r.two_m = x->two_m;
  r.fend = x->pend[slot];
  r.fcol = x->pcol[slot];
  r.fw = wk == W_UNIT ? nullptr : x->pw[slot];
  r.kin = x->rkin;
  r.elig = x->relig;
  r.chosen = x->rchosen;
  r.flag = x->flag;
  r.Cr = x->Cr;
  r.Sr = x->Sr;
  r.chunks = x->rchunks;
  r.chunk_cap = x->rchunk_cap;
  r.ctr = x->d_ctr;
  LV_CK(cudaMemsetAsync(x->rchosen, 0, (size_t)g.n, s));
  LV_CK(cudaMemsetAsync(x->recv, 0, (size_t)(g.n / 32 + 1) * sizeof(uint32_t), s));  // every refined community a singleton
  refine_rows(r, wk, x->num_sms, s);
  const GView f{g.n, g.begin, x->pend[slot], x->pcol[slot], r.fw};
  const uint32_t salt = bucket_salt(pass, 255, cfg.schedule_seed);
  const int rbuckets = kRefineBucketsPerB * cfg.buckets;  // fewer simultaneous decisions than local moving
  MoveArgs a{};
  a.g = f;
  a.Cp = x->Cr;
  a.K = x->K;
  a.Sigma = x->Sr;
  a.flag = x->flag;
  a.two_m = x->two_m;
  a.pickless = 0;
  a.salt = salt;
  a.nbuckets = (uint32_t)rbuckets;
  for (int k = 0; k < kMoveBins; ++k) a.bins[k] = x->bins[k];
  a.mv_vertex = x->mv_vertex;
  a.mv_target = x->mv_target;
  a.ctr = x->d_ctr;
  a.sched = x->sched;
  a.recv = x->recv;
  a.wide_spill = x->wide_spill;
  a.solo = pass > 0 || x->rows_unique;  // the filtered rows keep the rows' distinct columns
  a.refine = 1;
  BigArgs big{};
  big.g = f;
  big.Cp = x->Cr;
  big.items = x->bins[kBigBin];
  big.count = &x->d_ctr->bin_count[kBigBin];
  big.keyspace = g.n;
  big.ws = x->big;
  big.window = x->hub_window;
  big.rounds = x->hub_rounds;
  big.h_rounds = x->h_rounds;
  big.plan_done = x->plan_done;
  if (!x->pass_has_hubs) big.ws.slots = 0;  // filtered rows are no longer than the rows
  big.ctr = x->d_ctr;
  big.K = x->K;
  big.Sigma = x->Sr;
  big.flag = x->flag;
  big.two_m = x->two_m;
  big.pickless = 0;
  big.mv_vertex = x->mv_vertex;
  big.mv_target = x->mv_target;
  big.apply_Cp = x->Cr;
  big.apply_Sigma = x->Sr;
  big.accum_blocks = x->sched.move[kBigBin];
  for (int b = 0; b < rbuckets; ++b) {
    LV_CK(cudaMemsetAsync(x->d_ctr, 0, offsetof(Counters, it_gain_lo), s));
    a.bucket = (uint32_t)b;
    move_bucket(a, big, wk, x->num_sms, s, x->prof.mask ? &x->prof : nullptr, x->side.fork ? &x->side : nullptr);
    refine_resolve(r, x->mv_vertex, x->mv_target, x->recv, x->num_sms, s);
    refine_flags(r, salt, (uint32_t)rbuckets, (uint32_t)b, x->num_sms, s);
  }
  LV_CK(cudaGetLastError());
  return read_counters(x);  // hashtable and range errors of the refinement
}

louvain_status move_iteration(louvain_ctx *x, const GView &g, int wk, int pass, int t, bool skipping,
                              const Counters **h_out, bool completion) {
  const louvain_config &cfg = x->cfg;
  if (!completion) {
    louvain_status st = mark_iteration(x, pass, t);
    if (st) return st;
  }
  {
    const bool replay = x->sched.graphs && !x->graph_broken && !x->prof.mask && cfg.mode == LOUVAIN_MODE_PLAIN &&
                        !x->trace_x && !completion;  // graphs = 2 reaches here only when the phase graph is unusable
    louvain_status st0;
    if (replay && x->graph_pass != pass && (st0 = capture_iteration(x, g, wk, pass))) return st0;
    if (replay && !x->graph_broken) {
      const int rho = cfg.pickless_period;
      x->h_iter[0] = bucket_salt(pass, t, cfg.schedule_seed);
      x->h_iter[1] = (rho > 0 && ((t + rho / 2) % rho) == 0) ? 1u : 0u;
      LV_CK(cudaMemcpyAsync(x->d_iter, x->h_iter, 2 * sizeof(uint32_t), cudaMemcpyHostToDevice, x->stream));
      LV_CK(cudaGraphLaunch(x->gexec, x->stream));
      g_launches += x->graph_launches;
    } else if ((st0 = enqueue_iteration(x, g, wk, pass, t, skipping, nullptr, completion))) {
      return st0;
    }
    LV_CK(cudaGetLastError());
    if (x->batched)  // per-graph gain sums, read with the counters
      LV_CK(cudaMemcpyAsync(x->h_acc, x->b_acc, 2 * (size_t)x->G * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            x->stream));
    louvain_status st = read_counters(x);
    if (st) return st;
    record_iteration(x, g, pass, t, *x->h_ctr, completion);
    *h_out = x->h_ctr;
  }
  return LOUVAIN_OK;
}

// Exact modularity of `memb` on g (Eq. 1).  The lists of long rows go to
// rows[0..1] (g.n int32 each); by default two move-bin lists, which are free
// whenever modularity is computed.
louvain_status modularity_into(louvain_ctx *x, const GView &g, int wk, const int32_t *memb, const int64_t *sigma,
                               int64_t *sigma_scratch, i128 *num, i128 *den, int32_t *const *rows = nullptr) {
  LV_CK(cudaMemsetAsync(&x->d_ctr->q_sin, 0, 3 * sizeof(unsigned long long), x->stream));
  int32_t *warp_rows = rows ? rows[0] : x->bins[kBigBin];
  int32_t *block_rows = rows ? rows[1] : x->bins[kSpareBin];
  modularity_sums(g, wk, memb, sigma, sigma_scratch, warp_rows, block_rows, x->d_ctr, x->num_sms, x->stream);
  LV_CK(cudaGetLastError());
  louvain_status st = read_counters(x);
  if (st) return st;
  const Counters &h = *x->h_ctr;
  const i128 s_tot = ((i128)h.q_tot_hi << 32) + (i128)h.q_tot_lo;
  *num = (i128)x->two_m * (i128)h.q_sin - s_tot;
  *den = (i128)x->two_m * x->two_m;
  return LOUVAIN_OK;
}

// Resets the records of the previous run and starts the run's clock.
louvain_status begin_run(louvain_ctx *x) {
  const louvain_config &cfg = x->cfg;
  cudaStream_t s = x->stream;
  x->ran = false;
  x->graph_pass = -1;  // every pass captures its own iteration graph
  x->graph_broken = false;
  x->pexec_pass = -1;
  x->phase_broken = false;
  x->iter_stats.assign((size_t)std::max(cfg.max_passes, 1) * cfg.max_iterations * 4, 0);
  x->pass_stats.assign((size_t)std::max(cfg.max_passes, 1) * 6, 0);
  x->it_total = x->moves_total = x->evaluated_total = x->skipped_total = 0;
  x->learned_log.clear();
  for (int k = 0; k < K_NUM_KERNELS; ++k) {
    x->prof.ms[k] = 0;
    x->prof.launches[k] = 0;
    x->kbytes[k] = 0;
    x->kunits[k][0] = x->kunits[k][1] = 0;
  }
  x->prof.used = 0;
  for (auto &pt : x->timing) pt.timed = pt.aggregated = false;
  LV_CK(cudaEventRecord(x->run0, s));
  LV_CK(cudaMemsetAsync(x->d_ctr, 0, sizeof(Counters), s));
  return LOUVAIN_OK;
}

AggArgs agg_args(louvain_ctx *x, const GView &g, int wk, int slot) {
  AggArgs aa{};
  aa.sched = x->sched;
  aa.g = g;
  aa.wkind = wk;
  aa.Cp = x->Cp;
  aa.Sigma = x->Sigma;
  aa.Knew = x->Kalt;
  aa.cnt = x->cnt;
  aa.cdeg = x->cdeg;
  aa.newid = x->newid;
  aa.coff = x->coff;
  aa.hoff = x->hoff;
  aa.members = x->members;
  aa.kcoff = x->kcoff;
  aa.kcnt = x->kcnt;
  for (int k = 0; k < kNumBins; ++k) aa.mbins[k] = x->bins[k];
  aa.mbins[kMergeXlBin] = x->bins[kXlBin];
  aa.mbins[kMergeGroupBin] = x->bins[kGroupBin];
  aa.obegin = x->pbeg[slot];
  aa.oend = x->pend[slot];
  aa.ocol = x->pcol[slot];
  aa.ow = x->pw[slot];
  aa.mprefix = x->newid;  // free once the ids are relabelled
  aa.ctr = x->d_ctr;
  aa.scan_tmp = x->scan_tmp;
  return aa;
}

// Aggregation after the counts and ids (Algorithm 6): member lists, bins,
// dendrogram lookup and the merge into the other ping-pong CSR; g, wk, slot
// and nnzp then describe the super-vertex graph.
louvain_status aggregate(louvain_ctx *x, AggArgs &aa, int64_t gamma, PassTiming &pt, GView &g, int &wk, int &slot,
                         int64_t &nnzp) {
  cudaStream_t s = x->stream;
  louvain_status st;
  LV_CK(cudaMemsetAsync(&x->d_ctr->mbin_count[0], 0, sizeof(x->d_ctr->mbin_count), s));
  LV_CK(cudaMemsetAsync(&x->d_ctr->maxdeg, 0, 3 * sizeof(unsigned long long), s));
  x->prof.begin(K_SCATTER, s);
  agg_scatter_compact(aa, x->num_sms, s);
  x->prof.end(K_SCATTER, s);
  x->prof.begin(K_DENDRO, s);
  dendrogram_lookup(x->C, aa.Cp, x->n0, x->num_sms, s);
  x->prof.end(K_DENDRO, s);
  LV_CK(cudaGetLastError());
  if ((st = read_counters(x))) return st;
  int64_t mwindow = 0;
  int64_t mrounds = 0;
  if ((st = ensure_big_for(x, *x->h_ctr, x->h_ctr->maxdeg, (uint64_t)gamma, &mwindow, &mrounds))) return st;
  aa.big.window = mwindow;
  aa.big.rounds = mrounds;
  aa.big.accum_blocks = x->sched.merge[kBigBin];
  aa.big.h_rounds = x->h_rounds;
  aa.big.plan_done = x->plan_done;
  aa.big.g = g;
  aa.big.Cp = aa.Cp;
  aa.big.items = x->bins[kBigBin];
  aa.big.count = &x->d_ctr->mbin_count[kBigBin];
  aa.big.keyspace = gamma;
  aa.big.ws = x->big;
  if (x->h_ctr->big_items == 0) aa.big.ws.slots = 0;
  aa.big.ctr = x->d_ctr;
  aa.big.mprefix = aa.mprefix;
  aa.big.kcoff = x->kcoff;
  aa.big.kcnt = x->kcnt;
  aa.big.members = x->members;
  aa.big.obegin = aa.obegin;
  aa.big.oend = aa.oend;
  aa.big.ocol = aa.ocol;
  aa.big.ow = aa.ow;
  LV_CK(cudaMemsetAsync(&x->d_ctr->nnz_out, 0, sizeof(unsigned long long), s));
  LV_CK(cudaMemsetAsync(&x->d_ctr->mg_work[0][0], 0, sizeof(x->d_ctr->mg_work), s));
  agg_merge(aa, gamma, x->num_sms, s, x->prof.mask ? &x->prof : nullptr, x->side.fork ? &x->side : nullptr);
  LV_CK(cudaGetLastError());
  if ((st = read_counters(x))) return st;
  account_merge(x, *x->h_ctr);
  LV_CK(cudaEventRecord(pt.t2, s));
  pt.aggregated = true;
  nnzp = (int64_t)x->h_ctr->nnz_out;
  std::swap(x->K, x->Kalt);  // K of the super-vertices
  g = GView{gamma, x->pbeg[slot], x->pend[slot], x->pcol[slot], x->pw[slot]};
  wk = W_U32;
  slot ^= 1;
  return LOUVAIN_OK;
}

// Runs passes of Algorithm 1 from the start (fresh) or from where a
// suspended run stopped.  With budget > 0, a run that still has a pass to do
// after `budget` passes stops between two passes (*suspended = 1) and keeps
// its state for louvain_resume and louvain_save_state.
louvain_status run_impl(louvain_ctx *x, bool fresh = true, int32_t budget = 0, int32_t *suspended = nullptr) {
  const louvain_config &cfg = x->cfg;
  cudaStream_t s = x->stream;
  louvain_status st;
  const long long launches0 = g_launches;
  if (suspended) *suspended = 0;
  RunState &rs = x->rs;
  if (fresh) {
    x->suspended = false;
    x->launches = 0;
    if ((st = begin_run(x))) return st;
    rs.g = GView{x->n0, x->off0, x->off0 + 1, x->col0, x->w0};
    rs.wk = x->weighted ? W_U32 : W_UNIT;
    rs.slot = 0;
    rs.next_pass = 0;
    rs.nnzp = x->nnz0;
    rs.tau = cfg.tolerance;
    iota_i32(x->C, x->n0, x->num_sms, s);
  } else {
    if (!x->suspended) return LOUVAIN_E_STATE;
    x->suspended = false;
    x->graph_pass = -1;
    x->graph_broken = false;
    x->pexec_pass = -1;
    x->phase_broken = false;
    LV_CK(cudaEventRecord(x->run0, s));
  }
  if (x->big_dirty && x->big.slots > 0) {  // a failed run may have left table entries behind
    LV_CK(cudaMemsetAsync(x->big.tab, 0, (size_t)x->big.slots * sizeof(unsigned long long), s));
  }
  x->big_dirty = true;
  GView g = rs.g;
  int wk = rs.wk;
  double tau = rs.tau;
  bool pending = false, exhausted = true;
  int exit_reason = 0, passes = rs.next_pass, slot = rs.slot;
  int64_t nnzp = rs.nnzp;
  bool have_pass_state = false;
  for (int p = rs.next_pass; p < cfg.max_passes; ++p) {
    if (budget > 0 && p - rs.next_pass == budget) {  // stop between two passes
      rs = RunState{g, wk, slot, p, nnzp, tau};
      LV_CK(cudaStreamSynchronize(s));
      x->launches += g_launches - launches0;
      x->big_dirty = false;
      x->suspended = true;
      if (suspended) *suspended = 1;
      return LOUVAIN_OK;
    }
    PassTiming &pt = x->timing[p];
    LV_CK(cudaEventRecord(pt.t0, s));
    pt.timed = true;
    LV_CK(cudaMemsetAsync(&x->d_ctr->maxdeg, 0, sizeof(unsigned long long), s));
    x->cur_wbytes = wk == W_UNIT ? 0 : 4;
    LV_CK(cudaMemsetAsync(&x->d_ctr->big_slots, 0, 2 * sizeof(unsigned long long), s));
    x->prof.begin(K_PASS_INIT, s);
    {
      x->stamp = 0;  // pass init clears the stamps
      const LearnArgs L = learn_args(x, p, 0, false);
      pass_init(g, wk, p == 0, x->K, x->Sigma, x->Cp, x->flag, x->d_ctr, x->num_sms, s, &L, x->vbin, &x->sched);
      LV_CK(cudaMemsetAsync(x->recv, 0, (size_t)(g.n / 32 + 1) * sizeof(uint32_t), s));  // every community a singleton
      if (cfg.refine && p > 0)  // Leiden: the pass starts from the previous pass's P
        leiden_start(g.n, x->linit, x->K, x->Cp, x->Sigma, x->recv, x->num_sms, s);
    }
    x->prof.end(K_PASS_INIT, s);
    LV_CK(cudaGetLastError());
    if ((st = read_counters(x))) return st;
    x->pass_has_hubs = x->h_ctr->big_items > 0;
    if ((st = ensure_big_for(x, *x->h_ctr, x->h_ctr->maxdeg, (uint64_t)g.n, &x->hub_window, &x->hub_rounds)))
      return st;
    int li = 0;
    if ((st = move_phase(x, g, wk, p, tau, &li))) return st;
    have_pass_state = true;
    LV_CK(cudaEventRecord(pt.t1, s));
    ++passes;
    AggArgs aa = agg_args(x, g, wk, slot);
    x->prof.begin(K_COMM_COUNT, s);
    agg_count_scan(aa, x->num_sms, s);
    x->prof.end(K_COMM_COUNT, s);
    LV_CK(cudaGetLastError());
    if ((st = read_counters(x))) return st;
    const int64_t gamma = (int64_t)x->h_ctr->scan_total[0];
    aa.gamma = gamma;
    {
      int64_t *r = &x->pass_stats[(size_t)p * 6];
      r[0] = g.n;
      r[1] = nnzp;
      r[2] = li;
      r[3] = gamma;
      if (cfg.record_pass_modularity) {
        i128 qn, qd;
        if ((st = modularity_into(x, g, wk, x->Cp, x->Sigma, nullptr, &qn, &qd))) return st;
        put128(r + 4, qn);
      }
    }
    if (li <= 1) {  // globally converged
      pending = true;
      exhausted = false;
      exit_reason = 1;
      break;
    }
    // the partition to aggregate: C' (Louvain) or its refinement (Leiden)
    int64_t nagg = gamma;
    if (cfg.refine) {
      if ((st = refine_phase(x, g, wk, slot, p))) return st;
      aa.Cp = x->Cr;
      aa.Sigma = x->Sr;
      agg_count_scan(aa, x->num_sms, s);
      LV_CK(cudaGetLastError());
      if ((st = read_counters(x))) return st;
      nagg = (int64_t)x->h_ctr->scan_total[0];
      aa.gamma = nagg;  // the key space of the merge tables: the refined communities
    }
    if ((double)nagg / (double)g.n > cfg.aggregation_tolerance) {  // low shrink
      pending = true;
      exhausted = false;
      exit_reason = 2;
      break;
    }
    const int64_t n_before = g.n;
    if ((st = aggregate(x, aa, nagg, pt, g, wk, slot, nnzp))) return st;
    if (cfg.refine) leiden_next_init(n_before, x->Cp, x->Cr, x->lrep, x->linit, x->num_sms, s);
    tau /= cfg.tolerance_drop;
    have_pass_state = false;
  }
  (void)exhausted;
  if (pending) {
    dendrogram_lookup(x->C, x->Cp, x->n0, x->num_sms, s);
  } else {
    // identity memberships on the current graph (after max passes, or none)
    LV_CK(cudaMemsetAsync(&x->d_ctr->maxdeg, 0, sizeof(unsigned long long), s));
    pass_init(g, wk, passes == 0, x->K, x->Sigma, x->Cp, x->flag, x->d_ctr, x->num_sms, s);
    if (cfg.refine && passes > 0) {  // Leiden after the pass cap: the last pass's P, not its refinement
      leiden_start(g.n, x->linit, x->K, x->Cp, x->Sigma, x->recv, x->num_sms, s);
      dendrogram_lookup(x->C, x->Cp, x->n0, x->num_sms, s);
    }
    have_pass_state = true;
  }
  (void)have_pass_state;
  i128 qn = 0, qd = 0;
  x->prof.begin(K_MODULARITY, s);
  if ((st = modularity_into(x, g, wk, x->Cp, x->Sigma, nullptr, &qn, &qd))) return st;
  x->prof.end(K_MODULARITY, s);
  x->prof.begin(K_RENUMBER, s);
  renumber_dense(x->C, x->n0, x->n0, x->cnt, x->newid, x->scan_tmp, &x->d_ctr->scan_total[3], x->num_sms, s);
  x->prof.end(K_RENUMBER, s);
  LV_CK(cudaEventRecord(x->run1, s));
  LV_CK(cudaGetLastError());
  if ((st = read_counters(x))) return st;
  if (x->prof.mask) x->prof.collect();
  x->gamma = (int64_t)x->h_ctr->scan_total[3];
  x->trace_count = std::min<int64_t>((int64_t)x->h_ctr->trace_count, x->cfg.trace_capacity);
  x->qnum = qn;
  x->qden = qd;
  x->q = qd ? (double)qn / (double)qd : 0.0;
  x->passes = passes;
  x->exit_reason = exit_reason;
  float ms = 0;
  LV_CK(cudaEventElapsedTime(&ms, x->run0, x->run1));
  x->run_ms = ms;
  x->launches += g_launches - launches0;
  x->big_dirty = false;
  x->ran = true;
  return LOUVAIN_OK;
}

// Graphs of a batch that stop now (sel[g] = 1): exact modularity of each on
// the current union graph (Eq. 1 with the graph's own 2m) and its final
// memberships (dense ranks of the community ids of C' when newid is given,
// else of the current super-vertices).
louvain_status batch_finish(louvain_ctx *x, const GView &g, int wk, const int64_t *newid,
                            const std::vector<char> &sel) {
  cudaStream_t s = x->stream;
  const int64_t G = x->G;
  for (int64_t k = 0; k < G; ++k) x->h_flags[k] = sel[k] ? 1 : 0;
  LV_CK(cudaMemcpyAsync(x->b_sel, x->h_flags, (size_t)G, cudaMemcpyHostToDevice, s));
  unsigned long long *acc = x->b_acc + 3 * G;
  LV_CK(cudaMemsetAsync(acc, 0, 3 * (size_t)G * sizeof(unsigned long long), s));
  x->prof.begin(K_MODULARITY, s);
  batch_modularity(g, wk, x->b_gid, x->Cp, x->Sigma, x->b_sel, acc, acc + G, acc + 2 * G, x->num_sms, s);
  x->prof.end(K_MODULARITY, s);
  x->prof.begin(K_RENUMBER, s);
  batch_final(x->n0, x->C, x->b_ogid, x->Cp, newid, x->b_vo, x->b_sel, x->b_out, x->num_sms, s);
  x->prof.end(K_RENUMBER, s);
  LV_CK(cudaGetLastError());
  LV_CK(cudaMemcpyAsync(x->h_acc + 3 * G, acc, 3 * (size_t)G * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  LV_CK(cudaStreamSynchronize(s));
  for (int64_t k = 0; k < G; ++k) {
    if (!sel[k]) continue;
    const i128 tm = (i128)x->gtwo_m[k];
    const i128 sq = ((i128)x->h_acc[5 * G + k] << 32) + (i128)x->h_acc[4 * G + k];
    const i128 num = tm * (i128)x->h_acc[3 * G + k] - sq;
    const i128 den = tm * tm;
    int64_t *r = &x->b_results[(size_t)k * 8];
    put128(r + 2, num);
    put128(r + 4, den);
    x->b_q[k] = den ? (double)num / (double)den : 0.0;
  }
  return LOUVAIN_OK;
}

// Batched run: the pass loop of run_impl over the union of G graphs, with the
// iteration tolerance, the l_i <= 1 test and the aggregation tolerance taken
// per graph.  A graph that stops leaves the union at that pass's aggregation
// (its vertices get C' = -1 and are not renumbered); the remaining graphs
// are aggregated together.  Every graph sees exactly the sequence of states
// of a run on its own: the schedule hashes local vertex ids, and dense
// renumbering keeps each graph's super-vertices in order and contiguous.
louvain_status run_batched(louvain_ctx *x) {
  const louvain_config &cfg = x->cfg;
  cudaStream_t s = x->stream;
  louvain_status st;
  const long long launches0 = g_launches;
  if ((st = begin_run(x))) return st;
  const int64_t G = x->G;
  const int P = std::max(cfg.max_passes, 1);
  x->b_results.assign((size_t)G * 8, 0);
  x->b_q.assign((size_t)G, 0.0);
  x->b_passes.assign((size_t)G * P * 3, 0);
  for (int64_t k = 0; k < G; ++k) x->b_results[(size_t)k * 8 + 6] = x->gtwo_m[k];
  std::vector<int64_t> vo(x->vo0);
  std::vector<char> alive((size_t)G, 1), mv((size_t)G, 0), fin((size_t)G, 0);
  std::vector<int> li((size_t)G, 0);
  int64_t alive_count = G;
  LV_CK(cudaMemcpyAsync(x->b_vo, vo.data(), (size_t)(G + 1) * 8, cudaMemcpyHostToDevice, s));
  LV_CK(cudaMemcpyAsync(x->b_gid, x->b_ogid, (size_t)std::max<int64_t>(x->n0, 1) * 4, cudaMemcpyDeviceToDevice, s));

  GView g{x->n0, x->off0, x->off0 + 1, x->col0, x->w0};
  int wk = x->weighted ? W_U32 : W_UNIT;
  if (x->big_dirty && x->big.slots > 0) {
    LV_CK(cudaMemsetAsync(x->big.tab, 0, (size_t)x->big.slots * sizeof(unsigned long long), s));
  }
  x->big_dirty = true;
  iota_i32(x->C, x->n0, x->num_sms, s);
  double tau = cfg.tolerance;
  int passes = 0, slot = 0;
  int64_t nnzp = x->nnz0;
  for (int p = 0; p < cfg.max_passes && alive_count > 0; ++p) {
    PassTiming &pt = x->timing[p];
    LV_CK(cudaEventRecord(pt.t0, s));
    pt.timed = true;
    LV_CK(cudaMemsetAsync(&x->d_ctr->maxdeg, 0, sizeof(unsigned long long), s));
    x->cur_wbytes = wk == W_UNIT ? 0 : 4;
    LV_CK(cudaMemsetAsync(&x->d_ctr->big_slots, 0, 2 * sizeof(unsigned long long), s));
    x->prof.begin(K_PASS_INIT, s);
    pass_init(g, wk, p == 0, x->K, x->Sigma, x->Cp, x->flag, x->d_ctr, x->num_sms, s, nullptr, x->vbin, &x->sched);
    LV_CK(cudaMemsetAsync(x->recv, 0, (size_t)(g.n / 32 + 1) * sizeof(uint32_t), s));  // every community a singleton
    x->prof.end(K_PASS_INIT, s);
    LV_CK(cudaGetLastError());
    if ((st = read_counters(x))) return st;
    x->pass_has_hubs = x->h_ctr->big_items > 0;
    if ((st = ensure_big_for(x, *x->h_ctr, x->h_ctr->maxdeg, (uint64_t)g.n, &x->hub_window, &x->hub_rounds)))
      return st;
    // local-moving phase, each graph until its own tolerance test holds
    for (int64_t k = 0; k < G; ++k) {
      mv[k] = alive[k];
      li[k] = cfg.max_iterations;
      x->h_flags[k] = mv[k];
    }
    LV_CK(cudaMemcpyAsync(x->b_moving, x->h_flags, (size_t)G, cudaMemcpyHostToDevice, s));
    int li_union = 0;
    bool device_done = false;
    if (x->sched.graphs == 2 && !x->prof.mask && !x->phase_broken) {  // per-graph tests on the device
      for (int64_t k = 0; k < G; ++k) x->h_li[k] = cfg.max_iterations;
      LV_CK(cudaMemcpyAsync(x->b_li, x->h_li, (size_t)G * sizeof(int32_t), cudaMemcpyHostToDevice, s));
      if ((st = device_phase(x, g, wk, p, tau, &li_union))) return st;
      if (!x->phase_broken) {
        device_done = true;
        for (int64_t k = 0; k < G; ++k)
          if (mv[k]) li[k] = x->h_li[k];
      }
    }
    for (int t = 0; t < cfg.max_iterations && !device_done; ++t) {
      const Counters *h;
      if ((st = move_iteration(x, g, wk, p, t, false, &h))) return st;
      li_union = t + 1;
      bool any = false;
      for (int64_t k = 0; k < G; ++k) {
        if (!mv[k]) continue;
        const i128 gain = ((i128)x->h_acc[G + k] << 32) + (i128)x->h_acc[k];
        const i128 den2 = (i128)x->gtwo_m[k] * x->gtwo_m[k];
        const double total = den2 ? (double)(2 * gain) / (double)den2 : 0.0;
        if (total <= tau) {
          mv[k] = 0;
          li[k] = t + 1;
        } else {
          any = true;
        }
      }
      if (!any) break;
      for (int64_t k = 0; k < G; ++k) x->h_flags[k] = mv[k];
      LV_CK(cudaMemcpyAsync(x->b_moving, x->h_flags, (size_t)G, cudaMemcpyHostToDevice, s));
    }
    if (!device_done) {  // host-controlled iterations are timed one by one
      if ((size_t)p < x->iter_timed.size()) x->iter_timed[p] = 1;
      if ((st = mark_iteration(x, p, li_union))) return st;
    }
    LV_CK(cudaEventRecord(pt.t1, s));
    ++passes;
    AggArgs aa = agg_args(x, g, wk, slot);
    x->prof.begin(K_COMM_COUNT, s);
    agg_count_scan(aa, x->num_sms, s);
    x->prof.end(K_COMM_COUNT, s);
    batch_gather(x->newid, x->b_vo, G + 1, x->b_bound, s);
    LV_CK(cudaGetLastError());
    LV_CK(cudaMemcpyAsync(x->h_bound, x->b_bound, (size_t)(G + 1) * 8, cudaMemcpyDeviceToHost, s));
    if ((st = read_counters(x))) return st;
    int64_t gamma = (int64_t)x->h_ctr->scan_total[0];
    {
      int64_t *r = &x->pass_stats[(size_t)p * 6];
      r[0] = g.n;
      r[1] = nnzp;
      r[2] = li_union;
      r[3] = gamma;
    }
    // per-graph convergence (l_i <= 1) and aggregation tolerance tests
    int64_t nfin = 0;
    std::vector<int64_t> gam((size_t)G, 0);
    for (int64_t k = 0; k < G; ++k) {
      fin[k] = 0;
      if (!alive[k]) continue;
      const int64_t ng = vo[k + 1] - vo[k];
      gam[k] = x->h_bound[k + 1] - x->h_bound[k];
      int64_t *r = &x->b_passes[((size_t)k * P + p) * 3];
      r[0] = ng;
      r[1] = li[k];
      r[2] = gam[k];
      int why = 0;
      if (li[k] <= 1) why = 1;
      else if ((double)gam[k] / (double)ng > cfg.aggregation_tolerance) why = 2;
      if (why) {
        fin[k] = 1;
        ++nfin;
        int64_t *res = &x->b_results[(size_t)k * 8];
        res[0] = p + 1;
        res[1] = gam[k];
        res[7] = why;
      }
    }
    if (nfin) {
      if ((st = batch_finish(x, g, wk, x->newid, fin))) return st;
      for (int64_t k = 0; k < G; ++k)
        if (fin[k]) alive[k] = 0;
      alive_count -= nfin;
      if (alive_count == 0) break;
      // the finished graphs leave the union: recount without them
      batch_exclude(g.n, x->b_gid, x->b_sel, x->Cp, x->num_sms, s);
      agg_count_scan(aa, x->num_sms, s);
      LV_CK(cudaGetLastError());
      if ((st = read_counters(x))) return st;
      gamma = (int64_t)x->h_ctr->scan_total[0];
    }
    aa.gamma = gamma;
    // vertex offsets of the graphs in the super-vertex union
    std::vector<int64_t> nvo((size_t)G + 1, 0);
    for (int64_t k = 0; k < G; ++k) nvo[k + 1] = nvo[k] + (alive[k] ? gam[k] : 0);
    if (nvo[G] != gamma) {
      set_err(x, "batched aggregation: community counts do not add up (%lld vs %lld)", (long long)nvo[G],
              (long long)gamma);
      return LOUVAIN_E_STATE;
    }
    if ((st = aggregate(x, aa, gamma, pt, g, wk, slot, nnzp))) return st;
    vo.swap(nvo);
    LV_CK(cudaMemcpyAsync(x->b_vo, vo.data(), (size_t)(G + 1) * 8, cudaMemcpyHostToDevice, s));
    batch_gid(x->b_vo, G, g.n, x->b_gid, x->num_sms, s);
    LV_CK(cudaGetLastError());
    tau /= cfg.tolerance_drop;
  }
  if (alive_count > 0) {  // pass cap reached: identity memberships on the current graph
    LV_CK(cudaMemsetAsync(&x->d_ctr->maxdeg, 0, sizeof(unsigned long long), s));
    pass_init(g, wk, passes == 0, x->K, x->Sigma, x->Cp, x->flag, x->d_ctr, x->num_sms, s);
    for (int64_t k = 0; k < G; ++k) {
      if (!alive[k]) continue;
      int64_t *res = &x->b_results[(size_t)k * 8];
      res[0] = passes;
      res[1] = vo[k + 1] - vo[k];
      res[7] = 0;
    }
    if ((st = batch_finish(x, g, wk, nullptr, alive))) return st;
  }
  LV_CK(cudaEventRecord(x->run1, s));
  LV_CK(cudaGetLastError());
  if ((st = read_counters(x))) return st;
  if (x->prof.mask) x->prof.collect();
  int64_t total = 0;
  double qsum = 0;
  int maxp = 0;
  for (int64_t k = 0; k < G; ++k) {
    total += x->b_results[(size_t)k * 8 + 1];
    qsum += x->b_q[k];
    maxp = std::max<int>(maxp, (int)x->b_results[(size_t)k * 8]);
  }
  x->gamma = total;
  x->q = G ? qsum / (double)G : 0.0;
  x->qnum = x->qden = 0;
  x->passes = maxp;
  x->exit_reason = 0;
  float ms = 0;
  LV_CK(cudaEventElapsedTime(&ms, x->run0, x->run1));
  x->run_ms = ms;
  x->launches = g_launches - launches0;
  x->big_dirty = false;
  x->ran = true;
  return LOUVAIN_OK;
}

louvain_status ensure_prof_events(louvain_ctx *x) {
  if (!x->prof_events.empty()) return LOUVAIN_OK;
  x->prof_events.assign(512, nullptr);
  for (auto &e : x->prof_events)
    if (cudaEventCreate(&e)) {
      set_err(x, "event creation failed");
      return LOUVAIN_E_CUDA;
    }
  x->prof.pool = x->prof_events.data();
  x->prof.pool_size = (int)x->prof_events.size();
  return LOUVAIN_OK;
}

louvain_status validate_config(const louvain_config *c) {
  if (!c) return LOUVAIN_E_INVAL;
  if (c->max_passes < 0 || c->max_passes > 64 || c->max_iterations < 1 || c->max_iterations > 255) return LOUVAIN_E_INVAL;
  if (c->buckets < 1 || c->buckets > 65536 || c->pickless_period < 0) return LOUVAIN_E_INVAL;
  if (!(c->tolerance >= 0) || !(c->tolerance_drop > 0) || !(c->aggregation_tolerance >= 0)) return LOUVAIN_E_INVAL;
  if (c->mode != LOUVAIN_MODE_PLAIN && c->mode != LOUVAIN_MODE_LEARNED) return LOUVAIN_E_INVAL;
  if (c->mode == LOUVAIN_MODE_LEARNED && (!c->model || c->max_iterations > 127)) return LOUVAIN_E_INVAL;
  if (c->trace_capacity < 0 || c->learned_fallback < 0 || c->learned_fallback > 3) return LOUVAIN_E_INVAL;
  if (c->table_window < 0 || c->learned_min_degree < 0) return LOUVAIN_E_INVAL;
  if (c->asynchronous != 0 && c->asynchronous != 1) return LOUVAIN_E_INVAL;
  if (c->asynchronous && (c->mode != LOUVAIN_MODE_PLAIN || c->trace_capacity > 0)) return LOUVAIN_E_INVAL;
  if (c->refine != 0 && c->refine != 1) return LOUVAIN_E_INVAL;
  if (c->refine && (c->mode != LOUVAIN_MODE_PLAIN || c->asynchronous || c->trace_capacity > 0)) return LOUVAIN_E_INVAL;
  return LOUVAIN_OK;
}

// Host-side symmetry check: the multiset of entries (i, j, w) equals the
// multiset of their reversals (j, i, w).
bool host_symmetric(int64_t n, const int64_t *off, const int32_t *col, const int32_t *w) {
  struct E {
    int32_t a, b, w;
    bool operator<(const E &o) const { return a != o.a ? a < o.a : b != o.b ? b < o.b : w < o.w; }
    bool operator!=(const E &o) const { return a != o.a || b != o.b || w != o.w; }
  };
  std::vector<E> fwd, rev;
  fwd.reserve((size_t)off[n]);
  rev.reserve((size_t)off[n]);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = off[i]; k < off[i + 1]; ++k) {
      const int32_t ww = w ? w[k] : 1;
      fwd.push_back({(int32_t)i, col[k], ww});
      rev.push_back({col[k], (int32_t)i, ww});
    }
  std::sort(fwd.begin(), fwd.end());
  std::sort(rev.begin(), rev.end());
  for (size_t k = 0; k < fwd.size(); ++k)
    if (fwd[k] != rev[k]) return false;
  return true;
}

louvain_status create_impl(const louvain_graph *graph, const louvain_config *cfg, void *stream, louvain_ctx **out,
                            bool light = false, bool batched = false) {
  *out = nullptr;
  if (!graph || !cfg) {
    set_err(nullptr, "null graph or config");
    return LOUVAIN_E_INVAL;
  }
  if (validate_config(cfg)) {
    set_err(nullptr, "invalid configuration");
    return LOUVAIN_E_INVAL;
  }
  const int64_t n = graph->n, nnz = graph->nnz;
  if (n < 0 || nnz < 0 || n > INT32_MAX || (n > 0 && !graph->offsets) || (nnz > 0 && !graph->cols) ||
      (n == 0 && nnz != 0)) {
    set_err(nullptr, "bad graph sizes or pointers");
    return LOUVAIN_E_INVAL;
  }
  if (!graph->on_device && n > 0) {
    const int64_t *off = graph->offsets;
    if (off[0] != 0 || off[n] != nnz) {
      set_err(nullptr, "offsets[0] must be 0 and offsets[n] must equal nnz");
      return LOUVAIN_E_INVAL;
    }
    if (cfg->check_symmetry && !host_symmetric(n, off, graph->cols, graph->weights)) {
      set_err(nullptr, "graph is not symmetric (w_ij != w_ji)");
      return LOUVAIN_E_INVAL;
    }
  }
  louvain_ctx *x = new louvain_ctx();
  x->cfg = *cfg;
  x->stream = (cudaStream_t)stream;
  x->n0 = n;
  x->nnz0 = nnz;
  x->weighted = graph->weights != nullptr;
  auto fail = [&](louvain_status st) {
    g_create_err = x->err;
    louvain_destroy(x);
    return st;
  };
  if (cudaGetDevice(&x->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&x->num_sms, cudaDevAttrMultiProcessorCount, x->device) != cudaSuccess) {
    set_err(x, "no CUDA device");
    return fail(LOUVAIN_E_CUDA);
  }
  release_pool_threshold(x->device);
  louvain_status st;
  const int64_t nv = std::max<int64_t>(n, 1);
  // input graph
  if (graph->on_device) {
    x->off0 = graph->offsets;
    x->col0 = graph->cols;
    x->w0 = graph->weights;
  } else {
    int64_t *o;
    int32_t *c, *w = nullptr;
    if ((st = dalloc_n(x, &o, n + 1)) || (st = dalloc_n(x, &c, nnz))) return fail(st);
    if (x->weighted && (st = dalloc_n(x, &w, nnz))) return fail(st);
    if (n > 0 && cudaMemcpyAsync(o, graph->offsets, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, x->stream)) {
      set_err(x, "copy of offsets failed");
      return fail(LOUVAIN_E_CUDA);
    }
    if (nnz > 0 && cudaMemcpyAsync(c, graph->cols, (size_t)nnz * 4, cudaMemcpyHostToDevice, x->stream)) {
      set_err(x, "copy of cols failed");
      return fail(LOUVAIN_E_CUDA);
    }
    if (w && nnz > 0 && cudaMemcpyAsync(w, graph->weights, (size_t)nnz * 4, cudaMemcpyHostToDevice, x->stream)) {
      set_err(x, "copy of weights failed");
      return fail(LOUVAIN_E_CUDA);
    }
    x->off0 = o;
    x->col0 = c;
    x->w0 = w;
  }
  if (cudaMallocHost((void **)&x->h_ctr, sizeof(Counters)) != cudaSuccess) {
    set_err(x, "pinned allocation failed");
    return fail(LOUVAIN_E_NOMEM);
  }
  if ((st = dalloc(x, (void **)&x->d_ctr, sizeof(Counters)))) return fail(st);
  if (cudaMemsetAsync(x->d_ctr, 0, sizeof(Counters), x->stream)) return fail(LOUVAIN_E_CUDA);
  // validation and 2m
  if (n > 0) {
    LV_LAUNCH(k_validate_rows<<<grid_for(n, 256, x->num_sms, 8), 256, 0, x->stream>>>(n, x->off0, x->col0, x->d_ctr));
    if (nnz > 0)
      LV_LAUNCH(k_validate_entries<int32_t><<<grid_for(nnz, 256, x->num_sms, 8), 256, 0, x->stream>>>(nnz, n, x->col0, x->w0,
                                                                                            x->d_ctr));
    if (cudaGetLastError() != cudaSuccess) {
      set_err(x, "validation kernel failed to launch");
      return fail(LOUVAIN_E_CUDA);
    }
    if (graph->on_device) {
      int64_t ends[2];
      cudaMemcpyAsync(&ends[0], x->off0, 8, cudaMemcpyDeviceToHost, x->stream);
      cudaMemcpyAsync(&ends[1], x->off0 + n, 8, cudaMemcpyDeviceToHost, x->stream);
      if (cudaStreamSynchronize(x->stream) != cudaSuccess) {
        set_err(x, "stream error during validation");
        return fail(LOUVAIN_E_CUDA);
      }
      if (ends[0] != 0 || ends[1] != nnz) {
        set_err(x, "offsets[0] must be 0 and offsets[n] must equal nnz");
        return fail(LOUVAIN_E_INVAL);
      }
    }
    if (cudaMemcpyAsync(x->h_ctr, x->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, x->stream) ||
        cudaStreamSynchronize(x->stream)) {
      set_err(x, "stream error during validation");
      return fail(LOUVAIN_E_CUDA);
    }
    if (x->h_ctr->error & ERR_RANGE) {
      set_err(x, "malformed CSR: decreasing offsets, column out of range or non-positive weight");
      return fail(LOUVAIN_E_INVAL);
    }
    x->two_m = (long long)x->h_ctr->q_sin;
    x->rows_unique = x->h_ctr->descents[0] == x->h_ctr->descents[1];
    if (!batched && (unsigned long long)x->two_m >= (1ull << 32)) {  // a batch checks each graph's 2m
      set_err(x, "total weight 2m = %lld is 2^32 or more; int64 scores would overflow", x->two_m);
      return fail(LOUVAIN_E_OVERFLOW);
    }
  }
  if (light) {  // enough for louvain_modularity_of
    if (cudaStreamSynchronize(x->stream) != cudaSuccess) return fail(LOUVAIN_E_CUDA);
    *out = x;
    return LOUVAIN_OK;
  }
  // per-vertex state and work arrays
  if ((st = dalloc_n(x, &x->C, nv)) || (st = dalloc_n(x, &x->Cp, nv)) || (st = dalloc_n(x, &x->K, nv)) ||
      (st = dalloc_n(x, &x->Kalt, nv)) || (st = dalloc_n(x, &x->Sigma, nv)) || (st = dalloc_n(x, &x->flag, nv)) ||
      (st = dalloc_n(x, &x->vbin, nv)) || (st = dalloc_n(x, &x->recv, nv / 32 + 1)) ||
      (st = dalloc_n(x, &x->wide_spill, (int64_t)x->num_sms * kWideSpill)))
    return fail(st);
  if (cudaMemsetAsync(x->wide_spill, 0, (size_t)x->num_sms * kWideSpill * sizeof(unsigned long long), x->stream))
    return fail(LOUVAIN_E_CUDA);
  for (int k = 0; k < kMoveBins; ++k)
    if ((st = dalloc_n(x, &x->bins[k], nv))) return fail(st);
  if ((st = dalloc_n(x, &x->mv_vertex, nv)) || (st = dalloc_n(x, &x->mv_target, nv))) return fail(st);
  if ((st = dalloc_n(x, &x->cnt, nv)) || (st = dalloc_n(x, &x->cdeg, nv)) || (st = dalloc_n(x, &x->newid, nv + 1)) ||
      (st = dalloc_n(x, &x->coff, nv + 1)) || (st = dalloc_n(x, &x->hoff, nv + 1)) ||
      (st = dalloc_n(x, &x->kcoff, nv)) || (st = dalloc_n(x, &x->members, nv)) || (st = dalloc_n(x, &x->kcnt, nv)) ||
      (st = dalloc_n(x, &x->scan_tmp, (int64_t)scan_tmp_elems(nv))))
    return fail(st);
  for (int k = 0; k < 2; ++k)
    if ((st = dalloc_n(x, &x->pcol[k], nnz)) || (st = dalloc_n(x, &x->pw[k], nnz)) ||
        (st = dalloc_n(x, &x->pbeg[k], nv)) || (st = dalloc_n(x, &x->pend[k], nv)))
      return fail(st);
  if (cfg->mode == LOUVAIN_MODE_LEARNED || cfg->trace_capacity > 0) {
    // rows sampled for the feature x7 have at least dmin = max(min degree,
    // kSample + 1) entries, so no pass (whose nnz is at most the input's) has
    // more than nnz / dmin of them, nor more than nnz / kSampleChunk + nnz / dmin
    // chunks
    const int64_t dmin = std::max<int64_t>(cfg->learned_min_degree, kSample + 1);
    x->sample_cap = nnz / dmin + 1;
    x->chunk_cap = nnz / kSampleChunk + nnz / dmin + 1;
    if ((st = dalloc_n(x, &x->feat, nv)) || (st = dalloc_n(x, &x->seen, nv)) || (st = dalloc_n(x, &x->moved_at, nv)) ||
        (st = dalloc_n(x, &x->sample_at, nv)) || (st = dalloc_n(x, &x->sample, x->sample_cap * kSample)) ||
        (st = dalloc_n(x, &x->sample_n, x->sample_cap)) || (st = dalloc_n(x, &x->chunks, x->chunk_cap)))
      return fail(st);
  }
  if (cfg->refine) {
    x->rchunk_cap = nnz / kRefineChunk + nnz / (kRefineRowMax + 1) + 1;
    if ((st = dalloc_n(x, &x->Cr, nv)) || (st = dalloc_n(x, &x->Sr, nv)) || (st = dalloc_n(x, &x->relig, nv)) ||
        (st = dalloc_n(x, &x->rchosen, nv)) || (st = dalloc_n(x, &x->rkin, nv)) ||
        (st = dalloc_n(x, &x->rchunks, x->rchunk_cap)) || (st = dalloc_n(x, &x->linit, nv)) ||
        (st = dalloc_n(x, &x->lrep, nv)))
      return fail(st);
  }
  if (cfg->mode == LOUVAIN_MODE_LEARNED) {
    if ((st = dalloc_n(x, &x->cand, nv)) || (st = dalloc_n(x, &x->skip_list, nv)) ||
        (st = dalloc_n(x, &x->mlp, (int64_t)kMlpParams)))
      return fail(st);
    if (cudaMemcpyAsync(x->mlp, cfg->model, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, x->stream)) {
      set_err(x, "copy of the model parameters failed");
      return fail(LOUVAIN_E_CUDA);
    }
    x->model_hash = fnv1a_bytes(cfg->model, sizeof(float) * kMlpParams);
  }
  if (cfg->trace_capacity > 0) {
    if ((st = dalloc_n(x, &x->trace_x, cfg->trace_capacity * kFeatures)) ||
        (st = dalloc_n(x, &x->trace_y, cfg->trace_capacity)))
      return fail(st);
  }
  x->timing.resize((size_t)std::max(cfg->max_passes, 1));
  x->iter_ev.assign((size_t)std::max(cfg->max_passes, 1) * (cfg->max_iterations + 1), nullptr);
  x->iter_timed.assign((size_t)std::max(cfg->max_passes, 1), 0);
  for (auto &pt : x->timing) {
    if (cudaEventCreate(&pt.t0) || cudaEventCreate(&pt.t1) || cudaEventCreate(&pt.t2)) {
      set_err(x, "event creation failed");
      return fail(LOUVAIN_E_CUDA);
    }
  }
  if (cfg->profile_mask && ensure_prof_events(x)) return fail(LOUVAIN_E_CUDA);
  x->prof.mask = cfg->profile_mask;
  if (cudaEventCreate(&x->run0) || cudaEventCreate(&x->run1)) {
    set_err(x, "event creation failed");
    return fail(LOUVAIN_E_CUDA);
  }
  for (int k = 0; k < kSideStreams; ++k)
    if (cudaStreamCreateWithFlags(&x->side.s[k], cudaStreamNonBlocking) ||
        cudaEventCreateWithFlags(&x->side.join[k], cudaEventDisableTiming)) {
      set_err(x, "side stream creation failed");
      return fail(LOUVAIN_E_CUDA);
    }
  if (cudaEventCreateWithFlags(&x->side.fork, cudaEventDisableTiming)) {
    set_err(x, "event creation failed");
    return fail(LOUVAIN_E_CUDA);
  }
  if (cudaStreamSynchronize(x->stream) != cudaSuccess) {
    set_err(x, "stream error after allocation");
    return fail(LOUVAIN_E_CUDA);
  }
  *out = x;
  return LOUVAIN_OK;
}

template <typename T>
louvain_status pinned_n(louvain_ctx *x, T **p, int64_t n) {
  void *q = nullptr;
  if (cudaMallocHost(&q, (size_t)std::max<int64_t>(n, 1) * sizeof(T)) != cudaSuccess) {
    set_err(x, "pinned allocation of %lld bytes failed", (long long)(n * (int64_t)sizeof(T)));
    return LOUVAIN_E_NOMEM;
  }
  x->pinned.push_back(q);
  *p = (T *)q;
  return LOUVAIN_OK;
}

// Batch state on top of a context created for the union graph: vertex
// offsets, graph of each vertex, per-graph 2m (each must be below 2^32) and
// the check that no entry leaves its graph.
louvain_status setup_batch(louvain_ctx *x, const int64_t *vo, int64_t G) {
  cudaStream_t s = x->stream;
  louvain_status st;
  x->batched = true;
  x->G = G;
  x->vo0.assign(vo, vo + G + 1);
  const int64_t nv = std::max<int64_t>(x->n0, 1);
  if ((st = dalloc_n(x, &x->b_gid, nv)) || (st = dalloc_n(x, &x->b_ogid, nv)) || (st = dalloc_n(x, &x->b_out, nv)) ||
      (st = dalloc_n(x, &x->b_vo, G + 1)) || (st = dalloc_n(x, &x->b_bound, G + 1)) ||
      (st = dalloc_n(x, &x->b_two_m, G)) || (st = dalloc_n(x, &x->b_moving, G)) || (st = dalloc_n(x, &x->b_sel, G)) ||
      (st = dalloc_n(x, &x->b_acc, 6 * G)) || (st = dalloc_n(x, &x->b_li, G)) || (st = pinned_n(x, &x->h_li, G)))
    return st;
  if ((st = pinned_n(x, &x->h_acc, 6 * G)) || (st = pinned_n(x, &x->h_bound, G + 1)) ||
      (st = pinned_n(x, &x->h_flags, G)))
    return st;
  LV_CK(cudaMemcpyAsync(x->b_vo, vo, (size_t)(G + 1) * 8, cudaMemcpyHostToDevice, s));
  LV_CK(cudaMemsetAsync(x->b_two_m, 0, (size_t)G * sizeof(long long), s));
  LV_CK(cudaMemsetAsync(x->d_ctr, 0, sizeof(Counters), s));
  batch_gid(x->b_vo, G, x->n0, x->b_ogid, x->num_sms, s);
  const GView g0{x->n0, x->off0, x->off0 + 1, x->col0, x->w0};
  batch_check(g0, x->weighted ? W_U32 : W_UNIT, x->b_ogid, x->b_vo, x->b_two_m, x->d_ctr, x->num_sms, s);
  LV_CK(cudaGetLastError());
  x->gtwo_m.assign((size_t)G, 0);
  LV_CK(cudaMemcpyAsync(x->gtwo_m.data(), x->b_two_m, (size_t)G * sizeof(long long), cudaMemcpyDeviceToHost, s));
  if ((st = read_counters(x))) return st;
  if (x->h_ctr->error & ERR_RANGE) {
    set_err(x, "an entry of a graph's rows points outside the graph's vertex range");
    return LOUVAIN_E_INVAL;
  }
  for (int64_t k = 0; k < G; ++k)
    if ((unsigned long long)x->gtwo_m[k] >= (1ull << 32)) {
      set_err(x, "graph %lld: total weight 2m = %lld is 2^32 or more", (long long)k, x->gtwo_m[k]);
      return LOUVAIN_E_OVERFLOW;
    }
  x->bview.gid = x->b_gid;
  x->bview.vo = x->b_vo;
  x->bview.two_m = x->b_two_m;
  x->bview.moving = x->b_moving;
  x->bview.gain_lo = x->b_acc;
  x->bview.gain_hi = x->b_acc + G;
  x->bview.moves = x->b_acc + 2 * G;
  return LOUVAIN_OK;
}

}  // namespace

extern "C" {

void louvain_config_default(louvain_config *c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->max_passes = 10;
  c->max_iterations = 20;
  c->tolerance = 0.01;
  c->tolerance_drop = 10.0;
  c->aggregation_tolerance = 0.8;
  c->pickless_period = 4;
  c->buckets = 4;
  c->schedule_seed = 0;
  c->mode = LOUVAIN_MODE_PLAIN;
  c->model = nullptr;
  c->skip_threshold = 0.5f;
  c->record_pass_modularity = 0;
  c->check_symmetry = 0;
  c->profile_mask = 0;
  c->trace_capacity = 0;
  c->trace_rate = 1.0f;
  c->learned_fallback = 0;
  c->learned_skip_clears = 0;
  c->table_window = 0;
  c->asynchronous = 0;
  c->learned_min_degree = 0;
  c->refine = 0;
}

louvain_status louvain_create(const louvain_graph *graph, const louvain_config *cfg, void *stream, louvain_ctx **out) {
  if (!out) return LOUVAIN_E_INVAL;
  return create_impl(graph, cfg, stream, out);
}

louvain_status louvain_create_batched(const louvain_graph *graph, const int64_t *vertex_offsets, int64_t num_graphs,
                                      const louvain_config *cfg, void *stream, louvain_ctx **out) {
  if (!out) return LOUVAIN_E_INVAL;
  *out = nullptr;
  if (!graph || !cfg || !vertex_offsets || num_graphs < 1 || num_graphs > INT32_MAX) {
    set_err(nullptr, "null argument or bad number of graphs");
    return LOUVAIN_E_INVAL;
  }
  if (cfg->mode != LOUVAIN_MODE_PLAIN || cfg->trace_capacity != 0 || cfg->asynchronous || cfg->refine) {
    set_err(nullptr, "batched runs use the plain Louvain form without traces, on the deterministic schedule");
    return LOUVAIN_E_INVAL;
  }
  if (vertex_offsets[0] != 0 || vertex_offsets[num_graphs] != graph->n) {
    set_err(nullptr, "vertex_offsets[0] must be 0 and vertex_offsets[num_graphs] must equal n");
    return LOUVAIN_E_INVAL;
  }
  for (int64_t k = 0; k < num_graphs; ++k)
    if (vertex_offsets[k + 1] < vertex_offsets[k]) {
      set_err(nullptr, "vertex_offsets must not decrease");
      return LOUVAIN_E_INVAL;
    }
  louvain_ctx *x = nullptr;
  louvain_status st = create_impl(graph, cfg, stream, &x, false, true);
  if (st) return st;
  if ((st = setup_batch(x, vertex_offsets, num_graphs))) {
    g_create_err = x->err;
    louvain_destroy(x);
    return st;
  }
  *out = x;
  return LOUVAIN_OK;
}

louvain_status louvain_batch_results(const louvain_ctx *x, int64_t *results, double *q, int64_t *pass_records) {
  if (!x || !x->batched) return LOUVAIN_E_INVAL;
  if (!x->ran) return LOUVAIN_E_STATE;
  if (results) memcpy(results, x->b_results.data(), x->b_results.size() * sizeof(int64_t));
  if (q) memcpy(q, x->b_q.data(), x->b_q.size() * sizeof(double));
  if (pass_records && x->cfg.max_passes > 0)
    memcpy(pass_records, x->b_passes.data(), (size_t)x->G * x->cfg.max_passes * 3 * sizeof(int64_t));
  return LOUVAIN_OK;
}

louvain_status louvain_run(louvain_ctx *x) {
  if (!x) return LOUVAIN_E_INVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != x->device) cudaSetDevice(x->device);
  louvain_status st = x->batched ? run_batched(x) : run_impl(x);
  if (st != LOUVAIN_OK) x->ran = false;
  return st;
}

louvain_status louvain_run_passes(louvain_ctx *x, int32_t max_new_passes, int32_t *suspended) {
  if (!x || x->batched || x->cfg.refine) return LOUVAIN_E_INVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != x->device) cudaSetDevice(x->device);
  louvain_status st = run_impl(x, true, max_new_passes, suspended);
  if (st != LOUVAIN_OK) x->ran = x->suspended = false;
  return st;
}

louvain_status louvain_resume(louvain_ctx *x, int32_t max_new_passes, int32_t *suspended) {
  if (!x || x->batched) return LOUVAIN_E_INVAL;
  if (!x->suspended) return LOUVAIN_E_STATE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != x->device) cudaSetDevice(x->device);
  louvain_status st = run_impl(x, false, max_new_passes, suspended);
  if (st != LOUVAIN_OK) x->ran = x->suspended = false;
  return st;
}

namespace {

// Checkpoint layout: kCkptHeader int64 words, then the payload sections,
// each padded to 8 bytes (native byte order; the magic's bytes fail to match
// in the other order).
const char kCkptMagic[8] = {'L', 'V', 'C', 'K', 'P', 'T', '0', '1'};
constexpr int64_t kCkptHeader = 20;
enum CkptWord {
  CK_MAGIC = 0, CK_HEADER, CK_BYTES, CK_SUM, CK_N0, CK_NNZ0, CK_TWO_M, CK_WEIGHTED, CK_CONFIG, CK_PASS, CK_N, CK_NNZ,
  CK_TAU, CK_IT_TOTAL, CK_MOVES, CK_EVALUATED, CK_SKIPPED, CK_LEARNED_LOG
};

size_t pad8(size_t b) { return (b + 7) & ~(size_t)7; }

size_t ckpt_bytes(int64_t P, int64_t T, int64_t L, int64_t n0, int64_t n, int64_t nnz) {
  return 8 * (size_t)kCkptHeader + 8 * (size_t)(P * 6 + P * T * 4 + L * 3) + pad8(4 * (size_t)n0) +
         8 * (size_t)n + 8 * (size_t)(n + 1) + 2 * pad8(4 * (size_t)nnz);
}

// FNV-1a with 64-bit words as its symbols (the byte-wise constants, eight
// bytes per step): the payload checksum.
uint64_t fnv1a_words(const uint64_t *w, size_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= w[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

// Every setting that decides the remaining passes' results or the records.
uint64_t config_fingerprint(const louvain_ctx *x) {
  const louvain_config &c = x->cfg;
  const bool learned = c.mode == LOUVAIN_MODE_LEARNED;
  int64_t f[16] = {};
  f[0] = c.max_passes;
  f[1] = c.max_iterations;
  memcpy(&f[2], &c.tolerance, 8);
  memcpy(&f[3], &c.tolerance_drop, 8);
  memcpy(&f[4], &c.aggregation_tolerance, 8);
  f[5] = c.pickless_period;
  f[6] = c.buckets;
  f[7] = (int64_t)c.schedule_seed;
  f[8] = c.mode;
  f[9] = c.record_pass_modularity;
  f[14] = c.asynchronous + 2 * (int64_t)c.refine;
  if (learned) {
    memcpy(&f[10], &c.skip_threshold, 4);
    f[11] = c.learned_fallback;
    f[12] = c.learned_skip_clears;
    f[13] = (int64_t)x->model_hash;
    f[15] = c.learned_min_degree;
  }
  return fnv1a_bytes(f, sizeof f);
}

}  // namespace

louvain_status louvain_save_state(const louvain_ctx *xc, void *buf, size_t cap, size_t *size) {
  louvain_ctx *x = const_cast<louvain_ctx *>(xc);
  if (!x || x->batched) return LOUVAIN_E_INVAL;
  if (!x->suspended) return LOUVAIN_E_STATE;
  const RunState &rs = x->rs;
  const int64_t P = rs.next_pass, T = x->cfg.max_iterations, L = (int64_t)x->learned_log.size();
  const int64_t n = rs.g.n, nnz = rs.nnzp;
  const size_t need = ckpt_bytes(P, T, L, x->n0, n, nnz);
  if (size) *size = need;
  if (!buf) return LOUVAIN_OK;
  if (cap < need || ((uintptr_t)buf & 7)) {
    set_err(x, "checkpoint buffer must be 8-byte aligned and hold %zu bytes", need);
    return LOUVAIN_E_INVAL;
  }
  cudaStream_t s = x->stream;
  char *base = static_cast<char *>(buf);
  memset(base, 0, need);
  int64_t *h = reinterpret_cast<int64_t *>(base);
  memcpy(h, kCkptMagic, 8);
  h[CK_HEADER] = kCkptHeader;
  h[CK_BYTES] = (int64_t)need;
  h[CK_N0] = x->n0;
  h[CK_NNZ0] = x->nnz0;
  h[CK_TWO_M] = x->two_m;
  h[CK_WEIGHTED] = x->weighted;
  h[CK_CONFIG] = (int64_t)config_fingerprint(x);
  h[CK_PASS] = P;
  h[CK_N] = n;
  h[CK_NNZ] = nnz;
  memcpy(&h[CK_TAU], &rs.tau, 8);
  h[CK_IT_TOTAL] = x->it_total;
  h[CK_MOVES] = x->moves_total;
  h[CK_EVALUATED] = x->evaluated_total;
  h[CK_SKIPPED] = x->skipped_total;
  h[CK_LEARNED_LOG] = L;
  char *q = base + 8 * kCkptHeader;
  memcpy(q, x->pass_stats.data(), (size_t)P * 6 * 8);
  q += (size_t)P * 6 * 8;
  memcpy(q, x->iter_stats.data(), (size_t)P * T * 4 * 8);
  q += (size_t)P * T * 4 * 8;
  for (int64_t k = 0; k < L; ++k, q += 24) memcpy(q, x->learned_log[k].data(), 24);
  // dendrogram C[n0] and the super-vertex degrees K[n]
  if (x->n0) LV_CK(cudaMemcpyAsync(q, x->C, (size_t)x->n0 * 4, cudaMemcpyDeviceToHost, s));
  q += pad8((size_t)x->n0 * 4);
  if (n) LV_CK(cudaMemcpyAsync(q, x->K, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  q += (size_t)n * 8;
  // the super-vertex graph, compacted: its rows sit at the prefix of their
  // capacity bounds in one ping-pong buffer, and the device packs them into
  // the other one, which the next aggregation would write (free between
  // passes); the offsets are computed here from the row bounds
  std::vector<int64_t> b((size_t)n), e((size_t)n);
  if (n) {
    LV_CK(cudaMemcpyAsync(b.data(), rs.g.begin, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    LV_CK(cudaMemcpyAsync(e.data(), rs.g.end, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  }
  LV_CK(cudaStreamSynchronize(s));
  int64_t *off = reinterpret_cast<int64_t *>(q);
  off[0] = 0;
  for (int64_t i = 0; i < n; ++i) off[i + 1] = off[i] + (e[i] - b[i]);
  if (off[n] != nnz) {
    set_err(x, "suspended graph holds %lld entries, expected %lld", (long long)off[n], (long long)nnz);
    return LOUVAIN_E_STATE;
  }
  q += (size_t)(n + 1) * 8;
  int32_t *cols = reinterpret_cast<int32_t *>(q);
  uint32_t *wts = reinterpret_cast<uint32_t *>(q + pad8((size_t)nnz * 4));
  if (nnz) {
    const int free_slot = rs.slot;  // rs.g lives in the other buffer
    int64_t *d_off = x->hoff;        // aggregation scratch of n0 + 1 words, free between passes
    LV_CK(cudaMemcpyAsync(d_off, off, (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, s));
    LV_LAUNCH(k_compact_rows<<<grid_for(n * 32, 256, x->num_sms, 8), 256, 0, s>>>(
        n, rs.g.begin, rs.g.end, d_off, rs.g.col, static_cast<const uint32_t *>(rs.g.w), x->pcol[free_slot],
        x->pw[free_slot]));
    LV_CK(cudaGetLastError());
    LV_CK(cudaMemcpyAsync(cols, x->pcol[free_slot], (size_t)nnz * 4, cudaMemcpyDeviceToHost, s));
    LV_CK(cudaMemcpyAsync(wts, x->pw[free_slot], (size_t)nnz * 4, cudaMemcpyDeviceToHost, s));
    LV_CK(cudaStreamSynchronize(s));
  }
  h[CK_SUM] = (int64_t)fnv1a_words(reinterpret_cast<const uint64_t *>(base + 8 * kCkptHeader),
                                   (need - 8 * kCkptHeader) / 8);
  return LOUVAIN_OK;
}

louvain_status louvain_load_state(louvain_ctx *x, const void *buf, size_t size) {
  if (!x || x->batched || !buf || ((uintptr_t)buf & 7) || size < 8 * (size_t)kCkptHeader) return LOUVAIN_E_INVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != x->device) cudaSetDevice(x->device);
  const char *base = static_cast<const char *>(buf);
  const int64_t *h = reinterpret_cast<const int64_t *>(base);
  const louvain_config &cfg = x->cfg;
  auto refuse = [&](const char *why) {
    set_err(x, "checkpoint refused: %s", why);
    return LOUVAIN_E_INVAL;
  };
  x->ran = x->suspended = false;  // a refused checkpoint leaves neither results nor a suspended run
  if (memcmp(h, kCkptMagic, 8) || h[CK_HEADER] != kCkptHeader || h[CK_BYTES] != (int64_t)size)
    return refuse("not a checkpoint of this format, or truncated");
  if (h[CK_N0] != x->n0 || h[CK_NNZ0] != x->nnz0 || h[CK_TWO_M] != x->two_m || h[CK_WEIGHTED] != x->weighted)
    return refuse("taken on another input graph");
  if ((uint64_t)h[CK_CONFIG] != config_fingerprint(x)) return refuse("taken with another configuration or model");
  const int64_t P = h[CK_PASS], n = h[CK_N], nnz = h[CK_NNZ], L = h[CK_LEARNED_LOG], T = cfg.max_iterations;
  if (P < 1 || P >= cfg.max_passes || n < 1 || n > x->n0 || nnz < 0 || nnz > x->nnz0 || L < 0 || L > P)
    return refuse("sizes out of range");
  if (ckpt_bytes(P, T, L, x->n0, n, nnz) != size) return refuse("size does not match its header");
  if ((uint64_t)h[CK_SUM] !=
      fnv1a_words(reinterpret_cast<const uint64_t *>(base + 8 * kCkptHeader), (size - 8 * kCkptHeader) / 8))
    return refuse("checksum mismatch");
  double tau;
  memcpy(&tau, &h[CK_TAU], 8);
  if (!(tau >= 0) || !std::isfinite(tau)) return refuse("tolerance out of range");
  const char *q = base + 8 * kCkptHeader;
  const int64_t *pass_stats = reinterpret_cast<const int64_t *>(q);
  q += (size_t)P * 6 * 8;
  const int64_t *iter_stats = reinterpret_cast<const int64_t *>(q);
  q += (size_t)P * T * 4 * 8;
  const int64_t *llog = reinterpret_cast<const int64_t *>(q);
  q += (size_t)L * 24;
  const int32_t *C = reinterpret_cast<const int32_t *>(q);
  q += pad8((size_t)x->n0 * 4);
  const int64_t *K = reinterpret_cast<const int64_t *>(q);
  q += (size_t)n * 8;
  const int64_t *off = reinterpret_cast<const int64_t *>(q);
  q += (size_t)(n + 1) * 8;
  const int32_t *cols = reinterpret_cast<const int32_t *>(q);
  const uint32_t *wts = reinterpret_cast<const uint32_t *>(q + pad8((size_t)nnz * 4));
  // host checks: rows, dendrogram ids and degrees
  if (off[0] != 0 || off[n] != nnz) return refuse("row offsets do not span the entries");
  for (int64_t i = 0; i < n; ++i)
    if (off[i + 1] < off[i]) return refuse("decreasing row offsets");
  for (int64_t v = 0; v < x->n0; ++v)
    if (C[v] < 0 || C[v] >= n) return refuse("dendrogram id out of range");
  long long ksum = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (K[i] < 0 || K[i] > x->two_m) return refuse("vertex weight out of range");
    ksum += K[i];
  }
  if (ksum != x->two_m) return refuse("vertex weights do not sum to 2m");
  // restore into slot 0 of the ping-pong buffers, then check the entries
  cudaStream_t s = x->stream;
  LV_CK(cudaMemcpyAsync(x->C, C, (size_t)x->n0 * 4, cudaMemcpyHostToDevice, s));
  LV_CK(cudaMemcpyAsync(x->K, K, (size_t)n * 8, cudaMemcpyHostToDevice, s));
  LV_CK(cudaMemcpyAsync(x->pbeg[0], off, (size_t)n * 8, cudaMemcpyHostToDevice, s));
  LV_CK(cudaMemcpyAsync(x->pend[0], off + 1, (size_t)n * 8, cudaMemcpyHostToDevice, s));
  if (nnz) {
    LV_CK(cudaMemcpyAsync(x->pcol[0], cols, (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
    LV_CK(cudaMemcpyAsync(x->pw[0], wts, (size_t)nnz * 4, cudaMemcpyHostToDevice, s));
  }
  LV_CK(cudaMemsetAsync(x->d_ctr, 0, sizeof(Counters), s));
  if (nnz)
    LV_LAUNCH(k_validate_entries<uint32_t><<<grid_for(nnz, 256, x->num_sms, 8), 256, 0, s>>>(nnz, n, x->pcol[0],
                                                                                          x->pw[0], x->d_ctr));
  LV_CK(cudaGetLastError());
  LV_CK(cudaMemcpyAsync(x->h_ctr, x->d_ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s));
  LV_CK(cudaStreamSynchronize(s));
  if ((x->h_ctr->error & ERR_RANGE) || (long long)x->h_ctr->q_sin != x->two_m)
    return refuse("entries out of range, or weights that do not sum to 2m");
  LV_CK(cudaMemsetAsync(x->d_ctr, 0, sizeof(Counters), s));
  // records of the passes done, and the state the next pass starts from
  x->iter_stats.assign((size_t)cfg.max_passes * T * 4, 0);
  x->pass_stats.assign((size_t)cfg.max_passes * 6, 0);
  memcpy(x->pass_stats.data(), pass_stats, (size_t)P * 6 * 8);
  memcpy(x->iter_stats.data(), iter_stats, (size_t)P * T * 4 * 8);
  x->learned_log.assign((size_t)L, {});
  for (int64_t k = 0; k < L; ++k) memcpy(x->learned_log[k].data(), llog + 3 * k, 24);
  x->it_total = h[CK_IT_TOTAL];
  x->moves_total = h[CK_MOVES];
  x->evaluated_total = h[CK_EVALUATED];
  x->skipped_total = h[CK_SKIPPED];
  for (int k = 0; k < K_NUM_KERNELS; ++k) {
    x->prof.ms[k] = 0;
    x->prof.launches[k] = 0;
    x->kbytes[k] = 0;
    x->kunits[k][0] = x->kunits[k][1] = 0;
  }
  x->prof.used = 0;
  for (auto &pt : x->timing) pt.timed = pt.aggregated = false;
  x->launches = 0;
  x->graph_pass = -1;
  x->graph_broken = false;
  x->rs = RunState{GView{n, x->pbeg[0], x->pend[0], x->pcol[0], x->pw[0]}, W_U32, 1, (int)P, nnz, tau};
  x->suspended = true;
  return LOUVAIN_OK;
}

louvain_status louvain_modularity(const louvain_ctx *x, double *q, int64_t *num, int64_t *den) {
  if (!x || x->batched) return LOUVAIN_E_INVAL;  // a batch reports per graph (louvain_batch_results)
  if (!x->ran) return LOUVAIN_E_STATE;
  if (q) *q = x->q;
  if (num) put128(num, x->qnum);
  if (den) put128(den, x->qden);
  return LOUVAIN_OK;
}

louvain_status louvain_memberships(const louvain_ctx *xc, int32_t *out, int32_t out_on_device) {
  louvain_ctx *x = const_cast<louvain_ctx *>(xc);
  if (!x || (!out && x->n0 > 0)) return LOUVAIN_E_INVAL;
  if (!x->ran) return LOUVAIN_E_STATE;
  if (x->n0 == 0) return LOUVAIN_OK;
  LV_CK(cudaMemcpyAsync(out, x->batched ? x->b_out : x->C, (size_t)x->n0 * 4, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        x->stream));
  LV_CK(cudaStreamSynchronize(x->stream));
  return LOUVAIN_OK;
}

louvain_status louvain_records(const louvain_ctx *x, int64_t *iter_stats, int64_t *pass_stats, int64_t *summary) {
  if (!x) return LOUVAIN_E_INVAL;
  if (!x->ran) return LOUVAIN_E_STATE;
  const louvain_config &c = x->cfg;
  if (iter_stats && c.max_passes > 0)
    memcpy(iter_stats, x->iter_stats.data(), (size_t)c.max_passes * c.max_iterations * 4 * sizeof(int64_t));
  if (pass_stats && c.max_passes > 0) memcpy(pass_stats, x->pass_stats.data(), (size_t)c.max_passes * 6 * sizeof(int64_t));
  if (summary) {
    summary[0] = x->passes;
    summary[1] = x->gamma;
    put128(summary + 2, x->qnum);
    put128(summary + 4, x->qden);
    summary[6] = x->two_m;
    summary[7] = x->exit_reason;
  }
  return LOUVAIN_OK;
}

louvain_status louvain_stats(const louvain_ctx *xc, char *json, size_t cap) {
  louvain_ctx *x = const_cast<louvain_ctx *>(xc);
  if (!x || !json) return LOUVAIN_E_INVAL;
  if (!x->ran) return LOUVAIN_E_STATE;
  std::string s = "{";
  char buf[256];
  snprintf(buf, sizeof buf, "\"run_ms\": %.4f, \"passes\": %d, \"communities\": %lld, \"modularity\": %.12f, ",
           x->run_ms, x->passes, (long long)x->gamma, x->q);
  s += buf;
  snprintf(buf, sizeof buf,
           "\"iterations\": %lld, \"moves\": %lld, \"evaluated\": %lld, \"skipped\": %lld, \"device_bytes\": %zu, "
           "\"kernel_launches\": %lld, ",
           x->it_total, x->moves_total, x->evaluated_total, x->skipped_total, x->bytes, x->launches);
  s += buf;
  double tm = 0, ta = 0;
  std::string per = "\"per_pass\": [";
  for (int p = 0; p < x->passes; ++p) {
    float a = 0, b = 0;
    if (x->timing[p].timed) cudaEventElapsedTime(&a, x->timing[p].t0, x->timing[p].t1);
    if (x->timing[p].aggregated) cudaEventElapsedTime(&b, x->timing[p].t1, x->timing[p].t2);
    tm += a;
    ta += b;
    snprintf(buf, sizeof buf, "%s{\"move_ms\": %.4f, \"aggregate_ms\": %.4f, \"iteration_ms\": [", p ? ", " : "",
             a, b);
    per += buf;
    // local-moving time per iteration (completion steps included); a phase
    // under device control is one entry
    const int li = (int)x->pass_stats[(size_t)p * 6 + 2];
    const int steps = ((size_t)p < x->iter_timed.size() && x->iter_timed[p]) ? li : 1;
    const size_t base = (size_t)p * (x->cfg.max_iterations + 1);
    for (int t = 0; t < steps && x->timing[p].timed; ++t) {
      const size_t k0 = base + t, k1 = base + (steps == li ? t + 1 : li);
      float it = 0;
      if (k1 < x->iter_ev.size() && x->iter_ev[k0] && x->iter_ev[k1]) cudaEventElapsedTime(&it, x->iter_ev[k0], x->iter_ev[k1]);
      snprintf(buf, sizeof buf, "%s%.4f", t ? ", " : "", it);
      per += buf;
    }
    per += "]}";
  }
  per += "]";
  snprintf(buf, sizeof buf, "\"move_ms\": %.4f, \"aggregate_ms\": %.4f, \"other_ms\": %.4f, ", tm, ta,
           x->run_ms - tm - ta);
  s += buf;
  if (x->cfg.mode == LOUVAIN_MODE_LEARNED) {
    per += ", \"learned_passes\": [";
    for (size_t p = 0; p < x->learned_log.size(); ++p) {
      snprintf(buf, sizeof buf, "%s[%lld, %lld, %lld]", p ? ", " : "", x->learned_log[p][0], x->learned_log[p][1],
               x->learned_log[p][2]);
      per += buf;
    }
    per += "]";
  }
  s += per + ", \"kernels\": {";
  bool first = true;
  for (int k = 0; k < K_NUM_KERNELS; ++k) {
    if (x->prof.launches[k] == 0 && x->kbytes[k] == 0) continue;
    snprintf(buf, sizeof buf,
             "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"bytes\": %.0f, \"vertices\": %.0f, \"entries\": %.0f}",
             first ? "" : ", ", kKernelNames[k], x->prof.launches[k], x->prof.ms[k], x->kbytes[k], x->kunits[k][0],
             x->kunits[k][1]);
    s += buf;
    first = false;
  }
  s += "}}";
  if (s.size() + 1 > cap) return LOUVAIN_E_INVAL;
  memcpy(json, s.c_str(), s.size() + 1);
  return LOUVAIN_OK;
}

louvain_status louvain_set_profile(louvain_ctx *x, uint32_t mask) {
  if (!x) return LOUVAIN_E_INVAL;
  if (mask) {
    louvain_status st = ensure_prof_events(x);
    if (st) return st;
  }
  x->prof.mask = mask;
  x->cfg.profile_mask = mask;
  return LOUVAIN_OK;
}

// ---- launch schedule and autotuner

// Schedule words: group_max, warp_max, move blocks per SM of the bins
// (thread, warp, mid, block, hub, group), merge blocks per SM (thread, warp,
// mid, block, big), graphs.
static void sched_to_words(const Sched &s, int32_t *w) {
  int k = 0;
  w[k++] = s.group_max;
  w[k++] = s.half_max;
  w[k++] = s.warp_max;
  for (int b = 0; b < kMoveBins; ++b) w[k++] = s.move[b];
  for (int b = 0; b < kMergeBins; ++b) w[k++] = s.merge[b];
  w[k++] = s.graphs;
  w[k++] = s.concurrent;
}

static bool sched_from_words(const int32_t *w, Sched *s) {
  Sched t;
  int k = 0;
  t.group_max = w[k++];
  t.half_max = w[k++];
  t.warp_max = w[k++];
  for (int b = 0; b < kMoveBins; ++b) t.move[b] = w[k++];
  for (int b = 0; b < kMergeBins; ++b) t.merge[b] = w[k++];
  t.graphs = w[k++];
  t.concurrent = w[k++];
  if (t.group_max < kThreadMaxDeg || t.group_max > kGroupMaxDeg) return false;
  if (t.half_max < t.group_max || t.half_max > kHalfMaxDeg) return false;
  if (t.warp_max < t.half_max || t.warp_max > kWarpMaxDeg) return false;
  for (int b = 0; b < kMoveBins; ++b)
    if (t.move[b] < 1 || t.move[b] > 64) return false;
  for (int b = 0; b < kMergeBins; ++b)
    if (t.merge[b] < 1 || t.merge[b] > 64) return false;
  if (t.move[kBigBin] > 3 || t.merge[kBigBin] > 3) return false;  // accumulation: 3 blocks per SM at most
  if (t.graphs < 0 || t.graphs > 2) return false;
  if (t.concurrent != 0 && t.concurrent != 1) return false;
  *s = t;
  return true;
}

int32_t louvain_schedule_words(void) { return kSchedWords; }

louvain_status louvain_get_schedule(const louvain_ctx *x, int32_t *words, int32_t n) {
  if (!x || !words || n < kSchedWords) return LOUVAIN_E_INVAL;
  sched_to_words(x->sched, words);
  return LOUVAIN_OK;
}

louvain_status louvain_set_schedule(louvain_ctx *x, const int32_t *words, int32_t n) {
  if (!x || !words || n < kSchedWords) return LOUVAIN_E_INVAL;
  Sched s;
  if (!sched_from_words(words, &s)) {
    set_err(x, "schedule out of range");
    return LOUVAIN_E_INVAL;
  }
  x->sched = s;
  return LOUVAIN_OK;
}

// Autotuner: timed runs of the context's own graph choose the schedule.
// Results do not depend on the schedule, so every trial is a full run.
//   1. bin thresholds (group_max, warp_max): whole-run time of each pair;
//   2. blocks per SM: one run per candidate value with every bin set to it
//      and per-kernel event timing; each bin keeps its fastest value (the
//      bins' kernels are independent launches);
//   3. graph replay on or off: whole-run time.
// The tuned schedule is kept only if a final run beats the starting one.
louvain_status louvain_autotune(louvain_ctx *x, int32_t max_runs, char *json, size_t cap) {
  if (!x || max_runs < 1) return LOUVAIN_E_INVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != x->device) cudaSetDevice(x->device);
  const uint32_t mask0 = x->prof.mask;
  const Sched start = x->sched;
  int runs = 0;
  std::string trials;
  char buf[256];
  // whole-run trials keep the faster of two runs (run-to-run noise is a
  // few percent, about the size of the differences being judged)
  auto run_once = [&](const Sched &s, bool prof, double *ms) -> louvain_status {
    x->sched = s;
    louvain_status st;
    if (prof && (st = ensure_prof_events(x))) return st;
    x->prof.mask = prof ? (uint32_t)((1ull << K_NUM_KERNELS) - 1) : 0u;
    double best = 1e30;
    for (int rep = 0; rep < (prof ? 1 : 2); ++rep) {
      st = x->batched ? run_batched(x) : run_impl(x);
      if (st) break;
      best = std::min(best, x->run_ms);
    }
    x->prof.mask = mask0;
    ++runs;
    if (st) return st;
    *ms = best;
    return LOUVAIN_OK;
  };
  auto note = [&](const char *what, const Sched &s, double ms) {
    int32_t w[kSchedWords];
    sched_to_words(s, w);
    std::string ws;
    for (int k = 0; k < kSchedWords; ++k) ws += (k ? "," : "") + std::to_string(w[k]);
    snprintf(buf, sizeof buf, "%s{\"step\": \"%s\", \"ms\": %.4f, \"schedule\": [%s]}", trials.empty() ? "" : ", ",
             what, ms, ws.c_str());
    trials += buf;
  };
  louvain_status st;
  double ms = 0, start_ms = 0;
  if ((st = run_once(start, false, &ms))) goto fail;  // warm-up
  if ((st = run_once(start, false, &start_ms))) goto fail;
  note("start", start, start_ms);
  {
    Sched best = start;
    double best_ms = start_ms;
    // 1. thresholds (a half bin with half_max == group_max is empty).  The
    // triples differ by about as much as runs do, so a triple must beat the
    // current best by kMargin to replace it; otherwise noise alone would pick
    // a different triple, and different bins, from run to run.
    constexpr double kMargin = 0.015;
    const int gms[] = {16, 32, 48, 64};
    const int wms[] = {128, 256};
    for (int gm : gms)
      for (int hm : {gm, kHalfMaxDeg})
        for (int wm : wms) {
          if (wm < hm || runs >= max_runs) continue;
          if (gm == start.group_max && hm == start.half_max && wm == start.warp_max) continue;
          Sched t = best;
          t.group_max = gm;
          t.half_max = hm;
          t.warp_max = wm;
          if ((st = run_once(t, false, &ms))) goto fail;
          note("thresholds", t, ms);
          if (ms < best_ms * (1.0 - kMargin)) {
            best_ms = ms;
            best = t;
          }
        }
    // 2. blocks per SM, all bins at once per candidate; the current values
    // are measured first, so a bin keeps them unless a candidate is faster
    const int cands[] = {0, 2, 3, 4, 6, 8, 12, 16};  // 0: the current values
    double mv_best[kMoveBins], mg_best[kMergeBins];
    int mv_arg[kMoveBins], mg_arg[kMergeBins];
    for (int b = 0; b < kMoveBins; ++b) {
      mv_best[b] = 1e30;
      mv_arg[b] = best.move[b];
    }
    for (int b = 0; b < kMergeBins; ++b) {
      mg_best[b] = 1e30;
      mg_arg[b] = best.merge[b];
    }
    static const int mv_kid[kMoveBins] = {K_MOVE_THREAD, K_MOVE_WARP, K_MOVE_MID, K_MOVE_BLOCK, K_MOVE_HUB,
                                          K_MOVE_GROUP,  K_MOVE_XL,   -1,         K_MOVE_HALF};
    static const int mg_kid[kMergeBins] = {K_MERGE_THREAD, K_MERGE_WARP, K_MERGE_MID,   K_MERGE_BLOCK,
                                           K_MERGE_BIG,    K_MERGE_XL,   K_MERGE_GROUP};
    for (int v : cands) {
      if (runs >= max_runs) break;
      Sched t = best;
      if (v > 0) {
        for (int b = 0; b < kMoveBins; ++b) t.move[b] = b == kBigBin ? std::min(v, 3) : v;
        for (int b = 0; b < kMergeBins; ++b) t.merge[b] = b == kBigBin ? std::min(v, 3) : v;
      }
      if ((st = run_once(t, true, &ms))) goto fail;
      note(v > 0 ? "blocks" : "blocks current", t, ms);
      for (int b = 0; b < kMoveBins; ++b)
        if (mv_kid[b] >= 0 && x->prof.launches[mv_kid[b]] > 0 && x->prof.ms[mv_kid[b]] < mv_best[b]) {
          mv_best[b] = x->prof.ms[mv_kid[b]];
          mv_arg[b] = t.move[b];
        }
      for (int b = 0; b < kMergeBins; ++b)
        if (x->prof.launches[mg_kid[b]] > 0 && x->prof.ms[mg_kid[b]] < mg_best[b]) {
          mg_best[b] = x->prof.ms[mg_kid[b]];
          mg_arg[b] = t.merge[b];
        }
    }
    {
      Sched t = best;
      for (int b = 0; b < kMoveBins; ++b) t.move[b] = mv_arg[b];
      for (int b = 0; b < kMergeBins; ++b) t.merge[b] = mg_arg[b];
      if (runs < max_runs) {
        if ((st = run_once(t, false, &ms))) goto fail;
        note("blocks chosen", t, ms);
        if (ms < best_ms) {
          best_ms = ms;
          best = t;
        }
      }
    }
    // 3. concurrent bins, then graph replay
    if (runs < max_runs) {
      Sched t = best;
      t.concurrent = best.concurrent ? 0 : 1;
      if ((st = run_once(t, false, &ms))) goto fail;
      note("concurrent", t, ms);
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    for (int gm = 0; gm <= 2; ++gm) {  // graph replay: none, per iteration, whole phase under device control
      if (runs >= max_runs || gm == best.graphs) continue;
      Sched t = best;
      t.graphs = gm;
      if ((st = run_once(t, false, &ms))) goto fail;
      note("graphs", t, ms);
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    x->sched = best_ms < start_ms ? best : start;
    if (json) {
      int32_t w[kSchedWords];
      sched_to_words(x->sched, w);
      std::string ws;
      for (int k = 0; k < kSchedWords; ++k) ws += (k ? "," : "") + std::to_string(w[k]);
      std::string out = "{\"runs\": " + std::to_string(runs) + ", \"start_ms\": " + std::to_string(start_ms) +
                        ", \"tuned_ms\": " + std::to_string(std::min(best_ms, start_ms)) + ", \"schedule\": [" + ws +
                        "], \"trials\": [" + trials + "]}";
      if (out.size() + 1 > cap) return LOUVAIN_E_INVAL;
      memcpy(json, out.c_str(), out.size() + 1);
    }
  }
  // leave the context with a valid last run under the chosen schedule
  if ((st = run_once(x->sched, false, &ms))) goto fail;
  return LOUVAIN_OK;
fail:
  x->sched = start;
  x->prof.mask = mask0;
  x->ran = false;
  return st;
}

void louvain_destroy(louvain_ctx *x) {
  if (!x) return;
  for (void *p : x->allocs) cudaFreeAsync(p, x->stream);
  cudaStreamSynchronize(x->stream);
  for (auto &pt : x->timing) {
    if (pt.t0) cudaEventDestroy(pt.t0);
    if (pt.t1) cudaEventDestroy(pt.t1);
    if (pt.t2) cudaEventDestroy(pt.t2);
  }
  for (auto &e : x->prof_events)
    if (e) cudaEventDestroy(e);
  if (x->run0) cudaEventDestroy(x->run0);
  if (x->run1) cudaEventDestroy(x->run1);
  if (x->h_ctr) cudaFreeHost(x->h_ctr);
  if (x->h_rounds) cudaFreeHost(x->h_rounds);
  for (int k = 0; k < kSideStreams; ++k) {
    if (x->side.s[k]) cudaStreamDestroy(x->side.s[k]);
    if (x->side.join[k]) cudaEventDestroy(x->side.join[k]);
  }
  if (x->side.fork) cudaEventDestroy(x->side.fork);
  if (x->h_iter) cudaFreeHost(x->h_iter);
  if (x->gexec) cudaGraphExecDestroy(x->gexec);
  if (x->pexec) cudaGraphExecDestroy(x->pexec);
  for (cudaEvent_t e : x->iter_ev)
    if (e) cudaEventDestroy(e);
  if (x->h_phase) cudaFreeHost(x->h_phase);
  if (x->h_rec) cudaFreeHost(x->h_rec);
  if (x->plan_done) cudaEventDestroy(x->plan_done);
  for (void *p : x->pinned) cudaFreeHost(p);
  delete x;
}

const char *louvain_last_error(const louvain_ctx *x) {
  if (!x) return g_create_err.c_str();
  return x->err.c_str();
}

louvain_status louvain_modularity_of(const louvain_graph *graph, const int32_t *membership, void *stream, double *q,
                                     int64_t *num, int64_t *den) {
  if (!graph || !membership || graph->n < 0) return LOUVAIN_E_INVAL;
  louvain_config cfg;
  louvain_config_default(&cfg);
  cfg.max_passes = 0;
  louvain_ctx *x = nullptr;
  louvain_status st = create_impl(graph, &cfg, stream, &x, true);
  if (st) return st;
  const int64_t n = graph->n;
  const int32_t *memb = membership;
  int32_t *dm = nullptr;
  int64_t *sig = nullptr;
  if (!graph->on_device && n > 0) {
    if ((st = dalloc_n(x, &dm, n))) {
      louvain_destroy(x);
      return st;
    }
    cudaMemcpyAsync(dm, membership, (size_t)n * 4, cudaMemcpyHostToDevice, x->stream);
    memb = dm;
  }
  int32_t *rows = nullptr;
  if ((st = dalloc_n(x, &sig, std::max<int64_t>(n, 1))) || (st = dalloc_n(x, &rows, 2 * std::max<int64_t>(n, 1)))) {
    louvain_destroy(x);
    return st;
  }
  i128 qn = 0, qd = 0;
  GView g{n, x->off0, x->off0 + 1, x->col0, x->w0};
  int32_t *const lists[2] = {rows, rows + n};
  if (n > 0) st = modularity_into(x, g, x->weighted ? W_U32 : W_UNIT, memb, nullptr, sig, &qn, &qd, lists);
  if (!st && (x->h_ctr->error & ERR_MEMB)) {
    set_err(x, "membership id outside [0, n)");
    st = LOUVAIN_E_INVAL;
  }
  if (!st) {
    if (q) *q = qd ? (double)qn / (double)qd : 0.0;
    if (num) put128(num, qn);
    if (den) put128(den, qd);
  } else {
    g_create_err = x->err;
  }
  louvain_destroy(x);
  return st;
}

int64_t louvain_model_size(void) { return mlp_param_count(); }

louvain_status louvain_traces(const louvain_ctx *xc, float *features, float *labels, int64_t cap, int64_t *count,
                              int32_t on_device) {
  louvain_ctx *x = const_cast<louvain_ctx *>(xc);
  if (!x || !count || cap < 0) return LOUVAIN_E_INVAL;
  if (!x->ran) return LOUVAIN_E_STATE;
  const int64_t c = std::min(cap, x->trace_count);
  *count = c;
  if (c == 0) return LOUVAIN_OK;
  if (!features || !labels) return LOUVAIN_E_INVAL;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  LV_CK(cudaMemcpyAsync(features, x->trace_x, (size_t)c * kFeatures * sizeof(float), kind, x->stream));
  LV_CK(cudaMemcpyAsync(labels, x->trace_y, (size_t)c * sizeof(float), kind, x->stream));
  LV_CK(cudaStreamSynchronize(x->stream));
  return LOUVAIN_OK;
}

louvain_status louvain_mlp_forward(const float *params, const float *X, int64_t n, float *logits, void *stream) {
  if (!params || n < 0 || (n > 0 && (!X || !logits))) return LOUVAIN_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  mlp_forward(params, X, n, logits, s);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    g_create_err = "MLP forward kernel failed";
    return LOUVAIN_E_CUDA;
  }
  return LOUVAIN_OK;
}

louvain_status louvain_mlp_gradient(const float *params, const float *X, const float *Y, int64_t n, float *grad,
                                    float *loss, void *stream) {
  if (!params || !grad || n < 0 || (n > 0 && (!X || !Y))) return LOUVAIN_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (n > 0) {
    float *scratch = nullptr;
    if (cudaMallocAsync((void **)&scratch, sizeof(float) * mlp_grad_scratch_floats(n), s) != cudaSuccess) {
      cudaGetLastError();
      g_create_err = "allocation for the MLP gradient failed";
      return LOUVAIN_E_NOMEM;
    }
    mlp_gradient(params, X, Y, n, 1.0f / (float)n, grad, loss, scratch, s);
    cudaFreeAsync(scratch, s);
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    g_create_err = "MLP gradient kernel failed";
    return LOUVAIN_E_CUDA;
  }
  return LOUVAIN_OK;
}

louvain_status louvain_mlp_train(float *params, const float *X, const float *Y, int64_t n, int32_t epochs,
                                 int32_t batch, float lr, uint64_t seed, float *losses, void *stream) {
  if (!params || n <= 0 || !X || !Y || epochs < 0 || batch < 16 || !(lr > 0)) return LOUVAIN_E_INVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t b = std::min<int64_t>(batch, n);
  float *grad = nullptr, *m = nullptr, *v = nullptr, *Xb = nullptr, *Yb = nullptr, *lossd = nullptr, *scratch = nullptr;
  auto cleanup = [&]() {
    for (void *p : {(void *)grad, (void *)m, (void *)v, (void *)Xb, (void *)Yb, (void *)lossd, (void *)scratch})
      if (p) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
  };
  if (cudaMallocAsync((void **)&grad, sizeof(float) * kMlpParams, s) ||
      cudaMallocAsync((void **)&m, sizeof(float) * kMlpParams, s) ||
      cudaMallocAsync((void **)&v, sizeof(float) * kMlpParams, s) ||
      cudaMallocAsync((void **)&Xb, sizeof(float) * kFeatures * b, s) ||
      cudaMallocAsync((void **)&Yb, sizeof(float) * b, s) || cudaMallocAsync((void **)&lossd, sizeof(float), s) ||
      cudaMallocAsync((void **)&scratch, sizeof(float) * mlp_grad_scratch_floats(b), s)) {
    cudaGetLastError();
    cleanup();
    g_create_err = "allocation for MLP training failed";
    return LOUVAIN_E_NOMEM;
  }
  cudaMemsetAsync(m, 0, sizeof(float) * kMlpParams, s);
  cudaMemsetAsync(v, 0, sizeof(float) * kMlpParams, s);
  // a seeded visiting order: row r of an epoch is (offset + r) * stride mod n
  // with stride coprime to n (a permutation), fresh per epoch
  uint64_t state = seed ^ 0x9E3779B97F4A7C15ull;
  auto next = [&]() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  int step = 0;
  for (int e = 0; e < epochs; ++e) {
    uint64_t stride = (next() % (uint64_t)n) | 1ull;
    while (std::gcd(stride, (uint64_t)n) != 1) stride += 2;
    const uint64_t offset = next() % (uint64_t)n;
    cudaMemsetAsync(lossd, 0, sizeof(float), s);
    for (int64_t start = 0; start < n; start += b) {
      const int64_t cnt = std::min<int64_t>(b, n - start);
      mlp_gather_batch(X, Y, n, (int64_t)offset + start, cnt, stride, Xb, Yb, s);
      cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s);
      mlp_gradient(params, Xb, Yb, cnt, 1.0f / (float)cnt, grad, lossd, scratch, s);
      mlp_adam(params, grad, m, v, lr, ++step, s);
    }
    if (losses) {
      float l = 0;
      cudaMemcpyAsync(&l, lossd, sizeof(float), cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      losses[e] = l * (float)b / (float)n;
    }
  }
  const bool ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
  cleanup();
  if (!ok) {
    g_create_err = "MLP training kernels failed";
    return LOUVAIN_E_CUDA;
  }
  return LOUVAIN_OK;
}

const char *louvain_version(void) { return "gb300-louvain 0.1 (sm_103a)"; }

}  // extern "C"
