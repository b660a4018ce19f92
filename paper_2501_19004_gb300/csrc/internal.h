// Host-side declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace lv {

// Degree bins (entries per vertex when moving, per community when
// aggregating): a thread with registers up to kThreadMaxDeg entries, a warp
// with a shared-memory table up to kWarpMaxDeg, a 128-thread block up to
// kMidMaxDeg, a 512-thread block up to kBlockMaxDeg (shared tables of twice
// the entries), and beyond that chunks over the whole grid with global tables.
constexpr int kThreadMaxDeg = 16;
constexpr int kWarpMaxDeg = 256;
constexpr int kWarpCap = 512;       // >= 2 * kWarpMaxDeg, power of two
constexpr int kMidMaxDeg = 1024;
constexpr int kMidCap = 2048;
constexpr int kBlockMaxDeg = 4096;
constexpr int kBlockCap = 8192;
constexpr int kNumBins = 5;
constexpr int kBigBin = 4;

__host__ __device__ __forceinline__ int degree_bin(int64_t d) {
  return d <= kThreadMaxDeg ? 0 : d <= kWarpMaxDeg ? 1 : d <= kMidMaxDeg ? 2 : d <= kBlockMaxDeg ? 3 : 4;
}

// Local moving splits the warp bin: 16 < degree <= kGroupMaxDeg goes to
// groups of kGroupLanes lanes (several vertices per warp), the rest of the
// warp bin to whole warps.  The group bin is numbered after the others.
constexpr int kGroupLanes = 8;
constexpr int kGroupMaxDeg = 64;  // kGroupLanes lanes x 8 entries
constexpr int kGroupBin = 5;
// Local moving also splits the big bin: 4096 < degree <= kWideMaxDeg goes to
// the wide bin, one 1024-thread block with a 16384-slot shared table that
// holds only the entries whose community is not a known singleton (at most
// kWideCap distinct keys; beyond that the block's own global table of
// kWideSpill slots takes over); only larger degrees use the chunked global
// tables.  When aggregating, communities of total member degree (4096,
// kXlMaxDeg] take one 1024-thread block with a 16384-slot table (144 KB).
constexpr int kXlMaxDeg = 8192;
constexpr int kXlCap = 16384;
constexpr int kXlBin = 6;
constexpr int kWideMaxDeg = 32768;
constexpr int kWideCap = 12288;   // keys a wide vertex keeps in shared memory
constexpr int kWideSpill = 65536; // slots of a wide block's global table (2 x kWideMaxDeg)
// Bin 7 takes no vertices (its list serves as scratch for the modularity
// rows; its schedule word is kept so that schedules keep their layout).
constexpr int kSpareBin = 7;
// Degrees (group_max, half_max] go to groups of 16 lanes (two vertices per
// warp, rows of up to 128 entries).
constexpr int kHalfLanes = 16;
constexpr int kHalfMaxDeg = 128;
constexpr int kHalfBin = 8;
constexpr int kMoveBins = 9;
// Neighbour samples of the learned features: a row longer than kSample is
// represented by the neighbours j whose pair hash falls below
// 2^32 kSampleTarget / degree (about kSampleTarget of them, Binomial), stored
// in a block of kSample slots.  More than kSample of them (a chance below
// 1e-18 per row) and the row is read whole instead.  Rows are sampled in
// chunks of kSampleChunk entries, one block per chunk.
constexpr int kSample = 96;
constexpr int kSampleTarget = 32;
constexpr int kSampleChunk = 2048;
static_assert(sizeof(Counters::bin_count) == kMoveBins * sizeof(unsigned long long), "one counter per move bin");
// Aggregation bins: degree_bin's five plus communities with a total member
// degree in (4096, kXlMaxDeg] for one 1024-thread block (bin 5) and in
// (16, kGroupMaxDeg] for groups of kGroupLanes lanes (bin 6).
constexpr int kMergeXlBin = 5;
constexpr int kMergeGroupBin = 6;
constexpr int kMergeBins = 7;
__host__ __device__ __forceinline__ int merge_bin(int64_t d) {
  if (d > kThreadMaxDeg && d <= kGroupMaxDeg) return kMergeGroupBin;
  return (d > kBlockMaxDeg && d <= kXlMaxDeg) ? kMergeXlBin : degree_bin(d);
}

// Launch schedule of the binned kernels (louvain_autotune chooses one; the
// deterministic form's results never depend on it, since every bin's kernel
// computes the same exact decision for a vertex):
//   group_max  largest degree of the 8-lane group bin (16 = none, <= 64);
//   half_max   largest degree of the 16-lane group bin (>= group_max,
//              <= 128; = group_max for none);
//   warp_max   largest degree of the warp bin (>= half_max, <= 256); larger
//              degrees up to 1024 go to the 128-thread block bin;
//   move[b], merge[b]  blocks per SM of bin b's kernel (grid = SMs x blocks;
//              every kernel strides over its list, so any grid is correct);
//   graphs     1 = each iteration's launches are replayed from a CUDA graph;
//   concurrent 1 = a bucket's bin kernels run on side streams at the same
//              time (fork and join through events).
struct Sched {
  int group_max = kGroupMaxDeg;
  int half_max = kHalfMaxDeg;
  int warp_max = kWarpMaxDeg;
  int move[kMoveBins] = {2, 8, 12, 2, 3, 4, 1, 1, 4};  // thread, warp, mid, block, hub, group, xl, cluster, half
  int merge[kMergeBins] = {8, 8, 8, 2, 3, 1, 4};   // thread, warp, mid, block, big, xl, group
  int graphs = 0;
  int concurrent = 0;
};
constexpr int kSchedWords = 3 + kMoveBins + kMergeBins + 2;

// Flag byte of a vertex: kFlagUnproc = not processed since a neighbour moved
// (vertex pruning, Sec. 4.1.6).
constexpr uint8_t kFlagUnproc = 0x01;
constexpr unsigned long long kFlagUnproc8 = 0x0101010101010101ull;  // kFlagUnproc in each of 8 bytes

// Per-vertex byte of the pass (pass_init): the move bin in the low six bits
// (kVbinNone for degree 0) and kVbinTracked when the learned predictor keeps
// features for the vertex (degree at least its minimum; only then do
// neighbour moves count for it).
constexpr uint8_t kVbinBinMask = 0x3F;
constexpr uint8_t kVbinNone = 0x3F;
constexpr uint8_t kVbinTracked = 0x40;

// Side streams for concurrent bin kernels (created with the context).
constexpr int kSideStreams = 3;
struct SideStreams {
  cudaStream_t s[kSideStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSideStreams] = {};
};

__host__ __device__ __forceinline__ int move_bin(int64_t d, int group_max, int half_max, int warp_max) {
  if (d <= kThreadMaxDeg) return 0;
  if (d <= group_max) return kGroupBin;
  if (d <= half_max) return kHalfBin;
  if (d <= warp_max) return 1;
  if (d <= kMidMaxDeg) return 2;
  if (d <= kBlockMaxDeg) return 3;
  return d <= kWideMaxDeg ? kXlBin : kBigBin;
}

// Global tables of big items (hub vertices in local moving, communities with
// more than kBlockMaxDeg entries in aggregation).  Tables are kept empty
// between uses: the kernels that read a slot also clear it.
constexpr int kBigChunk = 4096;       // entries per accumulation chunk (512 threads x 8)
constexpr int kBigSmemSlots = 8192;   // shared pre-aggregation table per block
constexpr int kBigEvalSlots = 8192;   // occupied slots per evaluation block
struct BigWs {
  unsigned long long *tab = nullptr;  // packed slots (key + 1, weight); 0 = empty
  int64_t slots = 0;                  // capacity of tab
  int64_t *tot = nullptr;             // [items] entries of each item
  int64_t *toff = nullptr;            // [items+1] table offset
  int64_t *cpre = nullptr;            // [items+1] accumulation chunk prefix
  int64_t *epre = nullptr;            // [items+1] evaluation chunk prefix
  int32_t *occ = nullptr;             // [slots/2] occupied slots; item k's list starts at toff[k]/2
  unsigned long long *ocnt = nullptr; // [items] occupied slots per item
  long long *part_s = nullptr;        // [parts] partial argmax of an evaluation block
  int32_t *part_c = nullptr;
  unsigned long long *part_kid = nullptr;
  int64_t parts = 0;                  // capacity of part_*
  int64_t item_cap = 0;               // capacity of tot/toff/cpre/epre
  int64_t *rstart = nullptr;          // [round_cap + 2] first item of every round
  int64_t round_cap = 0;              // capacity of rstart (rounds)
  long long *nrounds = nullptr;       // [1] rounds the current items need (written by the plan)
};
// Items are processed in rounds: round r takes the items whose global table
// offset lies in [r * window, (r + 1) * window); the workspace holds window +
// the largest table, so every item of a round fits.  The plan kernel reports
// how many rounds the current items need, and only those are launched.

// Batched runs: many graphs as one union graph whose vertex ranges are the
// graphs (see batch.cu).  Null gid means a single graph.
struct BatchView {
  const int32_t *gid = nullptr;            // [n'] graph of each vertex
  const int64_t *vo = nullptr;             // [G+1] first vertex of each graph in the union
  const long long *two_m = nullptr;        // [G] total weight of each graph
  const int8_t *moving = nullptr;          // [G] 1 while the graph's moving phase runs
  unsigned long long *gain_lo = nullptr;   // [G] per-graph gain sums (low / high halves) and moves
  unsigned long long *gain_hi = nullptr;
  unsigned long long *moves = nullptr;
};

// 2m of vertex i's graph, and per-graph gain bookkeeping for a move.
__device__ __forceinline__ long long vertex_two_m(const BatchView &b, long long two_m, int32_t i) {
  return b.gid ? b.two_m[b.gid[i]] : two_m;
}
__device__ __forceinline__ void batch_gain(const BatchView &b, int32_t i, long long best_s, long long s_d) {
  if (!b.gid) return;
  const int32_t g = b.gid[i];
  const unsigned long long gain = (unsigned long long)best_s - (unsigned long long)s_d;
  atomicAdd(b.gain_lo + g, gain & 0xFFFFFFFFull);
  atomicAdd(b.gain_hi + g, gain >> 32);
  atomicAdd(b.moves + g, 1ull);
}

// Learned vertex-activity predictor and trace recorder (see mlp.cu).
struct LearnArgs {
  int enabled = 0;              // the predictor may skip flagged vertices
  int record = 0;               // per-vertex features are maintained
  const float *params = nullptr;  // device MLP parameters
  float4 *feat = nullptr;       // [n] intra fraction, margin, moved, valid
  // Neighbour-move feature (x7): bucket stamps, increasing within a pass
  // from 1 (0: never), and a hash-chosen sample of the neighbours of every
  // tracked vertex whose row is longer than kSample (shorter rows are their
  // own sample).
  uint32_t stamp = 0;             // stamp of the current bucket
  uint32_t *seen = nullptr;       // [n] stamp of the vertex's last evaluation
  uint32_t *moved_at = nullptr;   // [n] stamp of the bucket in which the vertex last moved
  int32_t *sample = nullptr;      // [sample_cap][kSample] samples (in no particular order)
  uint32_t *sample_n = nullptr;   // [sample_cap] neighbours that qualified for the block
  int32_t *sample_at = nullptr;   // [n] the vertex's sample block, -1: its row is its sample
  int64_t sample_cap = 0;         // sample blocks allocated
  int2 *chunks = nullptr;         // [chunk_cap] (vertex, chunk) of the rows to sample
  int64_t chunk_cap = 0;
  int32_t *cand = nullptr;      // [n] candidates of the bucket
  float thr_logit = 0.f;        // evaluate iff logit >= thr_logit
  int skip_clears = 0;          // a skip clears the flag (counts as "stay")
  int64_t min_degree = 0;       // only vertices of at least this degree are candidates and keep features
  int32_t *skip_list = nullptr; // [n] vertices skipped in the current iteration (count in ctr->skip_listed)
  const uint8_t *vbin = nullptr; // [n] per-vertex byte of the pass (kVbinTracked: features kept)
  float t_norm = 0.f, p_norm = 0.f;
  float *trace_x = nullptr;     // [cap][8] recorded features
  float *trace_y = nullptr;     // [cap] recorded labels (moved)
  int64_t trace_cap = 0;
  uint32_t trace_keep = 0;      // keep a decision iff hash16 < trace_keep
  uint32_t trace_salt = 0;
};

struct BigArgs {
  GView g;
  const int32_t *Cp;                  // C' (move: snapshot; merge: dense new ids)
  const int32_t *items;               // big item list (vertices or communities)
  const unsigned long long *count;    // its length (device)
  int64_t keyspace;                   // number of possible keys: n' or |Gamma|
  BigWs ws;
  int64_t window = 0;                 // table slots per round
  int accum_blocks = 3;               // blocks per SM of the accumulation kernel
  int64_t rounds = 1;                 // most rounds the items can need (rstart capacity)
  long long *h_rounds = nullptr;      // pinned host word: rounds needed (copied after the plan)
  cudaEvent_t plan_done = nullptr;    // recorded after that copy
  int static_rounds = 0;              // 1: launch all `rounds` rounds without asking (graph capture)
  Counters *ctr;
  // local moving
  const int64_t *K;
  const int64_t *Sigma;
  uint8_t *flag;
  long long two_m;
  int pickless;
  int32_t *mv_vertex;
  int32_t *mv_target;
  int async_apply = 0;                // asynchronous form: apply each move at its decision (emit_move)
  int32_t *apply_Cp = nullptr;        //   C' and Sigma' those moves write
  int64_t *apply_Sigma = nullptr;
  LearnArgs learn;
  BatchView batch;
  const uint32_t *iter = nullptr;     // graph replay: device words {salt, pickless} of the iteration
  // aggregation
  const int64_t *mprefix;             // member-degree exclusive prefix (community-vertex CSR order)
  const int64_t *kcoff;
  const int32_t *kcnt;
  const int32_t *members;
  const int64_t *obegin;
  int64_t *oend;
  int32_t *ocol;
  uint32_t *ow;
};

// big hub vertices of one bucket step / big communities of one aggregation
// (event timing: the accumulation kernel under K_MOVE_HUB / K_MERGE_BIG, the
// planning, evaluation and emission kernels under K_MOVE_HUB_EVAL /
// K_MERGE_BIG_EMIT)
struct KernelProf;
// Hub path of one bucket in two steps, so that the other bins' kernels run
// while the host waits for the number of rounds: big_move_plan (plan kernel
// and the copy of the round count), then big_move_rounds.
void big_move_plan(const BigArgs &b, cudaStream_t s, KernelProf *prof);
void big_move_rounds(const BigArgs &b, int wkind, int num_sms, cudaStream_t s, KernelProf *prof);
void big_merge(const BigArgs &b, int wkind, int num_sms, cudaStream_t s, KernelProf *prof);

inline int grid_for(int64_t n, int threads, int num_sms, int per_sm) {
  int64_t g = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

struct MoveArgs {
  GView g;
  int32_t *Cp;
  const int64_t *K;
  int64_t *Sigma;
  uint8_t *flag;
  long long two_m;
  int pickless;
  uint32_t salt;
  uint32_t nbuckets;
  uint32_t bucket;
  int32_t *bins[kMoveBins];
  int32_t *mv_vertex;
  int32_t *mv_target;
  Counters *ctr;
  LearnArgs learn;
  BatchView batch;
  Sched sched;
  const uint32_t *iter = nullptr;  // graph replay: device words {salt, pickless} of the iteration
  const uint8_t *vbin = nullptr;   // [n'] move bin of every vertex this pass (kVbinNone: degree 0), kVbinTracked bit
  int async_apply = 0;             // asynchronous form: movers apply their move at once (emit_move)
  // Known singletons (wide bin): bit c of `recv` is set once any vertex has
  // moved into community c this pass (k_apply sets it for every target).  A
  // neighbour j with C'[j] = j and bit j clear is alone in its community, so
  // with rows free of repeated columns (`solo`) its weight is K_{i->j}.
  uint32_t *recv = nullptr;        // [n'/32 + 1], cleared at every pass start
  int solo = 0;                    // 1: rows hold no repeated column and recv is maintained
  // Completion step of a learned iteration: the vertices of sel_list (count
  // *sel_count) are evaluated instead of a bucket's flagged vertices.
  const int32_t *sel_list = nullptr;
  const unsigned long long *sel_count = nullptr;
  unsigned long long *wide_spill = nullptr;  // [SMs][kWideSpill] global tables of the wide bin, kept empty
  int refine = 0;                  // Leiden refinement step: decisions only (refine_resolve applies them)
};

// Leiden refinement (refine.cu).  Rows of at most kRefineRowMax entries are
// filtered by one lane each; longer ones are cut into kRefineChunk-entry
// chunks, one warp each (at most nnz / kRefineChunk + nnz / (kRefineRowMax
// + 1) chunks).
constexpr int64_t kRefineRowMax = 16;
constexpr int kRefineChunk = 512;
// The filtered view of G' is
// GView{g.n, g.begin, fend, fcol, fw}: row i keeps its entries inside its
// community of P, at its own offsets.
struct RefineArgs {
  GView g;                      // current graph G'
  const int32_t *Cp;            // P (C' after local moving)
  const int64_t *K;             // vertex weights
  const int64_t *Sigma;         // Sigma' of P's communities
  long long two_m;
  int64_t *fend;                // [n] ends of the filtered rows
  int32_t *fcol;                // filtered entries (capacity: the ping-pong buffer)
  uint32_t *fw;                 // their weights, or null for unit weights
  unsigned long long *kin;      // [n] K_{i->C} of rows filtered in chunks
  uint8_t *elig;                // [n] well connected to its community of P
  uint8_t *chosen;              // [n] chosen as a target (no longer a singleton)
  uint8_t *flag;                // [n] move flags (kFlagUnproc: decides in its bucket)
  int32_t *Cr;                  // [n] refined partition
  int64_t *Sr;                  // [n] its community totals
  int2 *chunks;                 // chunk records (vertex, chunk) of long rows
  int64_t chunk_cap;
  Counters *ctr;
};
void refine_rows(const RefineArgs &r, int wkind, int num_sms, cudaStream_t s);
void refine_resolve(const RefineArgs &r, const int32_t *mv_vertex, const int32_t *mv_target, uint32_t *recv,
                    int num_sms, cudaStream_t s);
void refine_flags(const RefineArgs &r, uint32_t salt, uint32_t nbuckets, uint32_t bucket, int num_sms, cudaStream_t s);
void leiden_next_init(int64_t n, const int32_t *Cp, const int32_t *Cr, int32_t *rep, int32_t *init, int num_sms,
                      cudaStream_t s);
void leiden_start(int64_t n, const int32_t *init, const int64_t *K, int32_t *Cp, int64_t *Sigma, uint32_t *recv,
                  int num_sms, cudaStream_t s);

// Kernel identifiers for the optional per-kernel event timing.
enum KernelId : int {
  K_SELECT = 0, K_MOVE_THREAD, K_MOVE_WARP, K_MOVE_MID, K_MOVE_BLOCK, K_MOVE_HUB, K_APPLY, K_PASS_INIT,
  K_COMM_COUNT, K_SCATTER, K_MERGE_THREAD, K_MERGE_WARP, K_MERGE_MID, K_MERGE_BLOCK, K_MERGE_BIG, K_DENDRO,
  K_MODULARITY, K_RENUMBER, K_MOVE_HUB_EVAL, K_MERGE_BIG_EMIT, K_MLP_SELECT, K_MOVE_GROUP, K_MOVE_XL, K_MERGE_XL, K_MERGE_GROUP, K_MOVE_HALF, K_NUM_KERNELS
};
extern const char *const kKernelNames[K_NUM_KERNELS];

// Host-side event timing of selected kernels: a start and an end event
// around each launch whose id is in `mask`; collect() (after a stream
// synchronisation) adds the elapsed times up per kernel.
struct KernelProf {
  uint32_t mask = 0;
  cudaEvent_t *pool = nullptr;
  int pool_size = 0, used = 0;
  int pending_kid[256];
  double ms[K_NUM_KERNELS] = {};
  long long launches[K_NUM_KERNELS] = {};
  bool on(int kid) const { return (mask >> kid) & 1u; }
  void begin(int kid, cudaStream_t s) {
    if (!on(kid) || used + 2 > pool_size) return;
    pending_kid[used / 2] = kid;
    cudaEventRecord(pool[used++], s);
  }
  void end(int kid, cudaStream_t s) {
    if (!on(kid) || (used & 1) == 0) return;
    cudaEventRecord(pool[used++], s);
  }
  void collect() {
    for (int k = 0; k + 1 < used; k += 2) {
      float t = 0;
      cudaEventElapsedTime(&t, pool[k], pool[k + 1]);
      ms[pending_kid[k / 2]] += t;
      launches[pending_kid[k / 2]] += 1;
    }
    used = 0;
  }
};

// local-moving phase, one bucket step (select, decide per bin, apply)
void move_bucket(const MoveArgs &a, const BigArgs &big, int wkind, int num_sms, cudaStream_t s, KernelProf *prof,
                 const SideStreams *side = nullptr);

// pass initialisation: K (row sums on pass 0, else given), Sigma = K, C' = id,
// flags = 1, max degree into ctr->maxdeg; with vbin, every vertex's move
// bin under `sched` (0xFF for degree 0), read by the selection kernels
void pass_init(const GView &g, int wkind, int first_pass, int64_t *K, int64_t *Sigma, int32_t *Cp,
               uint8_t *flag, Counters *ctr, int num_sms, cudaStream_t s, const LearnArgs *learn = nullptr,
               uint8_t *vbin = nullptr, const Sched *sched = nullptr);

void iota_i32(int32_t *x, int64_t n, int num_sms, cudaStream_t s);
// every vertex unprocessed (the tracked bits kept)
void flag_all(uint8_t *flag, int64_t n, int num_sms, cudaStream_t s);

// aggregation phase
struct AggArgs {
  GView g;                  // G'
  int wkind;
  int32_t *Cp;              // C' (relabelled in place to new ids)
  const int64_t *Sigma;     // Sigma' after moving
  int64_t *Knew;            // [Gamma] K of the super-vertices
  unsigned long long *cnt;  // [n'] scratch: members per community
  unsigned long long *cdeg; // [n'] scratch: total degree per community
  int64_t *newid;           // [n'+1]
  int64_t *coff;            // [n'+1]
  int64_t *hoff;            // [n'+1]
  int32_t *members;         // [n']
  int64_t *kcoff;           // [Gamma]
  int32_t *kcnt;            // [Gamma]
  int32_t *mbins[kMergeBins]; // merge bins [Gamma] each
  // output super-vertex graph (holey CSR)
  int64_t *obegin;          // [Gamma]
  int64_t *oend;            // [Gamma]
  int32_t *ocol;
  uint32_t *ow;
  int64_t *mprefix;         // [n'] member-degree prefix (scratch)
  BigArgs big;
  Counters *ctr;
  long long *scan_tmp;      // block sums for the scans
  int64_t gamma;            // number of communities (keys of the merge tables)
  Sched sched;
};

// community sizes and degrees, scans; totals in ctr->scan_total[0..2]
// (Gamma, n', sum of degrees).
void agg_count_scan(const AggArgs &a, int num_sms, cudaStream_t s);
// member scatter + relabel C' to dense ids + per-community arrays + bins
void agg_scatter_compact(const AggArgs &a, int num_sms, cudaStream_t s);
// super-vertex rows (hash-merge of member rows); entries into ctr->nnz_out
void agg_merge(const AggArgs &a, int64_t gamma, int num_sms, cudaStream_t s, KernelProf *prof,
               const SideStreams *side = nullptr);

// C[v] = Cp[C[v]]
void dendrogram_lookup(int32_t *C, const int32_t *Cp, int64_t n, int num_sms, cudaStream_t s);

// exclusive scan of x (mode 0) or of [x > 0] (mode 1); total in *total
void scan_u64(const unsigned long long *in, int64_t *out, int64_t n, int mode, long long *tmp,
              unsigned long long *total, cudaStream_t s);

// modularity of membership `memb` on g: internal weight into ctr->q_sin and
// sum of Sigma_c^2 (split) into ctr->q_tot_lo/hi.  If sigma is null it is
// computed from the rows into sigma_scratch (zeroed here).  warp_rows and
// block_rows (g.n int32 each) receive the lists of long rows.
void modularity_sums(const GView &g, int wkind, const int32_t *memb, const int64_t *sigma,
                     int64_t *sigma_scratch, int32_t *warp_rows, int32_t *block_rows, Counters *ctr, int num_sms,
                     cudaStream_t s);

// order-preserving dense renumbering of x[0..n) with ids in [0, idspace);
// the number of distinct ids lands in *total
void renumber_dense(int32_t *x, int64_t n, int64_t idspace, unsigned long long *used, int64_t *newid,
                    long long *tmp, unsigned long long *total, int num_sms, cudaStream_t s);

// learned predictor (device pointers; see mlp.cu)
int64_t mlp_param_count();
void mlp_forward(const float *params, const float *X, int64_t n, float *logit, cudaStream_t s);
// gradient of the mean BCE added into grad (and the loss into *loss);
// scratch holds mlp_grad_scratch_floats(n) floats (per-block partials)
size_t mlp_grad_scratch_floats(int64_t n);
void mlp_gradient(const float *params, const float *X, const float *Y, int64_t n, float scale, float *grad,
                  float *loss, float *scratch, cudaStream_t s);
void mlp_adam(float *params, const float *grad, float *m, float *v, float lr, int step, cudaStream_t s);
void mlp_gather_batch(const float *X, const float *Y, int64_t n, int64_t start, int64_t count, uint64_t stride,
                      float *Xb, float *Yb, cudaStream_t s);

size_t scan_tmp_elems(int64_t n);

// batched runs (batch.cu)
void batch_gid(const int64_t *vo, int64_t G, int64_t n, int32_t *gid, int num_sms, cudaStream_t s);
void batch_check(const GView &g, int wkind, const int32_t *gid, const int64_t *vo, long long *two_m, Counters *ctr,
                 int num_sms, cudaStream_t s);
void batch_modularity(const GView &g, int wkind, const int32_t *gid, const int32_t *memb, const int64_t *sigma,
                      const int8_t *sel, unsigned long long *sin, unsigned long long *lo, unsigned long long *hi,
                      int num_sms, cudaStream_t s);
void batch_gather(const int64_t *src, const int64_t *idx, int64_t m, int64_t *out, cudaStream_t s);
void batch_final(int64_t n0, int32_t *C, const int32_t *ogid, const int32_t *Cp, const int64_t *newid,
                 const int64_t *vo, const int8_t *fin, int32_t *out, int num_sms, cudaStream_t s);
void batch_exclude(int64_t n, const int32_t *gid, const int8_t *fin, int32_t *Cp, int num_sms, cudaStream_t s);

// Kernel launches issued by this thread since the last reset (the library's
// own kernels only; memsets and copies are not counted).
extern thread_local long long g_launches;
#define LV_LAUNCH(...) (++::lv::g_launches, __VA_ARGS__)
#define LV_TIMED(prof, kid, s, ...)          \
  do {                                       \
    if (prof) (prof)->begin((kid), (s));     \
    LV_LAUNCH(__VA_ARGS__);                  \
    if (prof) (prof)->end((kid), (s));       \
  } while (0)

}  // namespace lv
