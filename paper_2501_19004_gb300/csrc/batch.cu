// Batched runs on sm_103a: many independent graphs as one union graph whose
// vertex ranges are the graphs.  Every graph keeps the semantics of a run of
// its own (paper Algorithm 1 / 4 per graph): its own 2m in Eq. 2, its own
// gain sum, iteration count, convergence and aggregation tests, and bucket
// hashes of its local vertex ids.  Passes run in lockstep; a graph that stops
// gets its final memberships and modularity at that moment and leaves the
// union.  The kernels below build the union and keep the per-graph books.
#include "internal.h"
#include "tables.cuh"

namespace lv {
namespace {

__global__ void k_batch_gid(const int64_t *vo, int64_t G, int64_t n, int32_t *gid) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    gid[i] = (int32_t)upper_index(vo, G, i);
}

// Every entry of a graph's rows must stay inside the graph (else ERR_RANGE);
// the row weights are summed into the graph's 2m.  Warp per vertex.
template <int WK>
__global__ void k_batch_check(GView g, const int32_t *gid, const int64_t *vo, long long *two_m, Counters *ctr) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  bool bad = false;
  for (int64_t i = warp; i < g.n; i += nw) {
    const int32_t gg = gid[i];
    const int64_t lo = vo[gg], hi = vo[gg + 1];
    unsigned long long k = 0;
    for (int64_t e = g.begin[i] + lane; e < g.end[i]; e += 32) {
      const int32_t c = g.col[e];
      if (c < lo || c >= hi) bad = true;
      k += load_w<WK>(g.w, e);
    }
    k = warp_sum_u(k);
    if (lane == 0 && k) atomicAdd((unsigned long long *)two_m + gg, k);
  }
  if (bad) atomicOr(&ctr->error, (unsigned long long)ERR_RANGE);
}

// Per-graph modularity sums (Eq. 1) of the graphs with sel[g] != 0: internal
// weight (warp per vertex) and sum of Sigma_c^2 (split in 32-bit halves).
template <int WK>
__global__ void k_batch_mod_rows(GView g, const int32_t *gid, const int32_t *memb, const int8_t *sel,
                                 unsigned long long *sin) {
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int64_t i = warp; i < g.n; i += nw) {
    const int32_t gg = gid[i];
    if (!sel[gg]) continue;
    const int32_t ci = memb[i];
    unsigned long long in = 0;
    for (int64_t e = g.begin[i] + lane; e < g.end[i]; e += 32)
      if (memb[__ldg(g.col + e)] == ci) in += load_w<WK>(g.w, e);
    in = warp_sum_u(in);
    if (lane == 0 && in) atomicAdd(sin + gg, in);
  }
}

__global__ void k_batch_sigma_sq(const int64_t *sigma, const int32_t *gid, int64_t n, const int8_t *sel,
                                 unsigned long long *lo, unsigned long long *hi) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t gg = gid[c];  // community ids are vertex ids of the same graph
    if (!sel[gg]) continue;
    const unsigned long long s = (unsigned long long)sigma[c];
    if (!s) continue;
    const unsigned long long sq = s * s;
    atomicAdd(lo + gg, sq & 0xFFFFFFFFull);
    atomicAdd(hi + gg, sq >> 32);
  }
}

__global__ void k_batch_gather(const int64_t *src, const int64_t *idx, int64_t m, int64_t *out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = src[idx[k]];
}

// Final memberships of the graphs that stop now (fin[g] = 1): dense ids in
// [0, |Gamma_g|) from the order-preserving ranks of the raw C' ids (newid);
// their C entries are then frozen (-1).  With newid == nullptr (after the
// pass cap) the ids are the current super-vertices.
__global__ void k_batch_final(int64_t n0, int32_t *C, const int32_t *ogid, const int32_t *Cp, const int64_t *newid,
                              const int64_t *vo, const int8_t *fin, int32_t *out) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = C[v];
    if (x < 0) continue;
    const int32_t g = ogid[v];
    if (!fin[g]) continue;
    out[v] = newid ? (int32_t)(newid[Cp[x]] - newid[vo[g]]) : (int32_t)(x - vo[g]);
    C[v] = -1;
  }
}

__global__ void k_batch_exclude(int64_t n, const int32_t *gid, const int8_t *fin, int32_t *Cp) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (fin[gid[i]]) Cp[i] = -1;
}

}  // namespace

void batch_gid(const int64_t *vo, int64_t G, int64_t n, int32_t *gid, int num_sms, cudaStream_t s) {
  if (n <= 0) return;
  LV_LAUNCH(k_batch_gid<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(vo, G, n, gid));
}

void batch_check(const GView &g, int wkind, const int32_t *gid, const int64_t *vo, long long *two_m, Counters *ctr,
                 int num_sms, cudaStream_t s) {
  if (g.n <= 0) return;
  if (wkind == W_UNIT)
    LV_LAUNCH(k_batch_check<W_UNIT><<<grid_for(g.n * 32, 256, num_sms, 16), 256, 0, s>>>(g, gid, vo, two_m, ctr));
  else
    LV_LAUNCH(k_batch_check<W_U32><<<grid_for(g.n * 32, 256, num_sms, 16), 256, 0, s>>>(g, gid, vo, two_m, ctr));
}

void batch_modularity(const GView &g, int wkind, const int32_t *gid, const int32_t *memb, const int64_t *sigma,
                      const int8_t *sel, unsigned long long *sin, unsigned long long *lo, unsigned long long *hi,
                      int num_sms, cudaStream_t s) {
  if (g.n <= 0) return;
  if (wkind == W_UNIT)
    LV_LAUNCH(k_batch_mod_rows<W_UNIT><<<grid_for(g.n * 32, 256, num_sms, 16), 256, 0, s>>>(g, gid, memb, sel, sin));
  else
    LV_LAUNCH(k_batch_mod_rows<W_U32><<<grid_for(g.n * 32, 256, num_sms, 16), 256, 0, s>>>(g, gid, memb, sel, sin));
  LV_LAUNCH(k_batch_sigma_sq<<<grid_for(g.n, 256, num_sms, 16), 256, 0, s>>>(sigma, gid, g.n, sel, lo, hi));
}

void batch_gather(const int64_t *src, const int64_t *idx, int64_t m, int64_t *out, cudaStream_t s) {
  if (m <= 0) return;
  LV_LAUNCH(k_batch_gather<<<(int)((m + 255) / 256), 256, 0, s>>>(src, idx, m, out));
}

void batch_final(int64_t n0, int32_t *C, const int32_t *ogid, const int32_t *Cp, const int64_t *newid,
                 const int64_t *vo, const int8_t *fin, int32_t *out, int num_sms, cudaStream_t s) {
  if (n0 <= 0) return;
  LV_LAUNCH(k_batch_final<<<grid_for(n0, 256, num_sms, 16), 256, 0, s>>>(n0, C, ogid, Cp, newid, vo, fin, out));
}

void batch_exclude(int64_t n, const int32_t *gid, const int8_t *fin, int32_t *Cp, int num_sms, cudaStream_t s) {
  if (n <= 0) return;
  LV_LAUNCH(k_batch_exclude<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(n, gid, fin, Cp));
}

}  // namespace lv
