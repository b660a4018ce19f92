// Host-side declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace lv {

// Degree bins of the local-moving phase: a thread per vertex up to
// kThreadMaxDeg entries, a warp with a shared-memory table up to
// kWarpMaxDeg, a block with a shared-memory table up to kBlockMaxDeg, and a
// block with a global-memory table beyond (hubs).
constexpr int kThreadMaxDeg = 16;
constexpr int kWarpMaxDeg = 256;
constexpr int kWarpCap = 512;       // >= 2 * kWarpMaxDeg, power of two
constexpr int kBlockMaxDeg = 4096;
constexpr int kBlockCap = 8192;     // >= 2 * kBlockMaxDeg, power of two
constexpr int kNumBins = 4;

// Global hashtable workspace for hub vertices / large communities: each
// block of the hub kernels owns one slice of `slice` slots.
struct HubWs {
  int32_t *keys = nullptr;
  unsigned long long *vals = nullptr;
  int64_t slice = 0;   // slots per block
  int blocks = 0;      // number of slices
};

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
  int32_t *bins[kNumBins];
  int32_t *mv_vertex;
  int32_t *mv_target;
  HubWs ws;
  Counters *ctr;
  // learned mode (null when plain)
  const float *mlp;          // device parameters
  float *feat;               // per-vertex features [n][8]
  float skip_threshold;
  int learned;
};

// local-moving phase, one bucket step (select, decide per bin, apply)
void move_bucket(const MoveArgs &a, int wkind, int num_sms, cudaStream_t s);

// pass initialisation: K (row sums on pass 0, else given), Sigma = K, C' = id,
// flags = 1, max degree into ctr->maxdeg
void pass_init(const GView &g, int wkind, int first_pass, int64_t *K, int64_t *Sigma, int32_t *Cp,
               uint8_t *flag, Counters *ctr, int num_sms, cudaStream_t s);

void iota_i32(int32_t *x, int64_t n, int num_sms, cudaStream_t s);

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
  int32_t *mbins[kNumBins]; // merge bins [Gamma] each
  // output super-vertex graph (holey CSR)
  int64_t *obegin;          // [Gamma]
  int64_t *oend;            // [Gamma]
  int32_t *ocol;
  int64_t *ow;
  HubWs ws;
  Counters *ctr;
  long long *scan_tmp;      // block sums for the scans
  int64_t gamma;            // number of communities (keys of the merge tables)
};

// community sizes and degrees, scans; totals in ctr->scan_total[0..2]
// (Gamma, n', sum of degrees).
void agg_count_scan(const AggArgs &a, int num_sms, cudaStream_t s);
// member scatter + relabel C' to dense ids + per-community arrays + bins
void agg_scatter_compact(const AggArgs &a, int num_sms, cudaStream_t s);
// super-vertex rows (hash-merge of member rows); entries into ctr->nnz_out
void agg_merge(const AggArgs &a, int64_t gamma, int num_sms, cudaStream_t s);

// C[v] = Cp[C[v]]
void dendrogram_lookup(int32_t *C, const int32_t *Cp, int64_t n, int num_sms, cudaStream_t s);

// exclusive scan of x (mode 0) or of [x > 0] (mode 1); total in *total
void scan_u64(const unsigned long long *in, int64_t *out, int64_t n, int mode, long long *tmp,
              unsigned long long *total, cudaStream_t s);

// modularity of membership `memb` on g: internal weight into ctr->q_sin and
// sum of Sigma_c^2 (split) into ctr->q_tot_lo/hi.  If sigma is null it is
// computed from the rows into sigma_scratch (zeroed here).
void modularity_sums(const GView &g, int wkind, const int32_t *memb, const int64_t *sigma,
                     int64_t *sigma_scratch, Counters *ctr, int num_sms, cudaStream_t s);

// order-preserving dense renumbering of x[0..n) with ids in [0, idspace);
// the number of distinct ids lands in *total
void renumber_dense(int32_t *x, int64_t n, int64_t idspace, unsigned long long *used, int64_t *newid,
                    long long *tmp, unsigned long long *total, int num_sms, cudaStream_t s);

// learned predictor
int64_t mlp_param_count();
void mlp_features_init(float *feat, int64_t n, int num_sms, cudaStream_t s);

size_t scan_tmp_elems(int64_t n);

}  // namespace lv
