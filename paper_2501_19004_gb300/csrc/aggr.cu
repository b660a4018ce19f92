// Aggregation phase of the Louvain method on sm_103a (arXiv 2501.19004,
// Sec. 4.2.3 Algorithm 3 and its GPU form Algorithm 6), the renumbering and
// dendrogram lookup of the pass loop (Algorithm 1 / 4), and modularity (Eq. 1).
//
// Aggregation, per pass:
//   k_comm_count     community sizes and total degrees (countCommunityVertices
//                    and communityTotalDegree), warp-aggregated atomics;
//   scans            order-preserving new ids, member offsets and the holey
//                    row offsets of the super-vertex graph (exclusiveScan);
//   k_comm_scatter   community-vertex CSR G'_{C'} and relabelling of C';
//   k_comm_compact   per-super-vertex arrays, K of the super-vertices
//                    (= Sigma' of the communities) and merge bins;
//   k_merge_*        one super-vertex row per community: scanCommunities with
//                    self = true over all member rows into a table, emitted
//                    into the holey row (thread / warp / block / global bins).
#include <climits>

#include "internal.h"

namespace lv {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

int grid_for(int64_t n, int threads, int num_sms, int per_sm) {
  int64_t g = (n + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

// --------------------------------------------------------------- count
__global__ void __launch_bounds__(256) k_comm_count(GView g, const int32_t *Cp, unsigned long long *cnt,
                                                    unsigned long long *cdeg) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool ok = i < g.n;
    const int32_t c = ok ? Cp[i] : -1;
    const unsigned long long deg = ok ? (unsigned long long)(g.end[i] - g.begin[i]) : 0ull;
    const unsigned peers = __match_any_sync(kFull, c);
    unsigned long long sum = 0;
    for (unsigned m = peers; m; m &= m - 1) sum += __shfl_sync(peers, deg, __ffs(m) - 1);
    if (ok && lane == __ffs(peers) - 1) {
      atomicAdd(cnt + c, (unsigned long long)__popc(peers));
      if (sum) atomicAdd(cdeg + c, sum);
    }
  }
}

// --------------------------------------------------------------- scan
constexpr int kScanNT = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanNT * kScanItems;

template <int MODE>
__device__ __forceinline__ long long scan_in(const unsigned long long *in, int64_t i, int64_t n) {
  if (i >= n) return 0;
  const unsigned long long v = in[i];
  return MODE == 0 ? (long long)v : (long long)(v != 0);
}

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *total) {
  __shared__ long long wsum[kScanNT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < kScanNT / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanNT / 32) wsum[lane] = w;
  }
  __syncthreads();
  const long long before = warp > 0 ? wsum[warp - 1] : 0;
  *total = wsum[kScanNT / 32 - 1];
  __syncthreads();
  return before + x - v;
}

template <int MODE>
__global__ void __launch_bounds__(kScanNT) k_scan_reduce(const unsigned long long *in, int64_t n, long long *bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) s += scan_in<MODE>(in, base + k * kScanNT + threadIdx.x, n);
  long long tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanNT) k_scan_blocks(long long *bsum, int64_t nb, unsigned long long *total) {
  long long carry = 0;
  for (int64_t base = 0; base < nb; base += kScanNT) {
    const int64_t i = base + threadIdx.x;
    const long long v = i < nb ? bsum[i] : 0;
    long long tot;
    const long long ex = block_exclusive_scan(v, &tot);
    if (i < nb) bsum[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) *total = (unsigned long long)carry;
}

template <int MODE>
__global__ void __launch_bounds__(kScanNT) k_scan_down(const unsigned long long *in, int64_t *out, int64_t n,
                                                       const long long *bsum) {
  __shared__ long long tile[kScanTile];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) tile[k * kScanNT + threadIdx.x] = scan_in<MODE>(in, base + k * kScanNT + threadIdx.x, n);
  __syncthreads();
  long long loc[kScanItems];
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    loc[k] = s;
    s += tile[threadIdx.x * kScanItems + k];
  }
  long long tot;
  const long long ex = block_exclusive_scan(s, &tot) + bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) tile[threadIdx.x * kScanItems + k] = ex + loc[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t i = base + k * kScanNT + threadIdx.x;
    if (i < n) out[i] = tile[k * kScanNT + threadIdx.x];
  }
}

__global__ void k_write_total(int64_t *out, int64_t n, const unsigned long long *total) { out[n] = (int64_t)*total; }

// --------------------------------------------------------------- scatter
__global__ void __launch_bounds__(256) k_comm_scatter(int64_t n, int32_t *Cp, unsigned long long *cursor,
                                                      const int64_t *coff, const int64_t *newid, int32_t *members) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool ok = i < n;
    const int32_t c = ok ? Cp[i] : -1;
    const unsigned peers = __match_any_sync(kFull, c);
    const int leader = __ffs(peers) - 1;
    unsigned long long top = 0;
    if (ok && lane == leader) top = atomicAdd(cursor + c, (unsigned long long)__popc(peers));
    top = __shfl_sync(kFull, top, leader);
    if (ok) {
      const unsigned long long pos = top + __popc(peers & lanemask_lt());
      members[coff[c] + (int64_t)pos] = (int32_t)i;
      Cp[i] = (int32_t)newid[c];
    }
  }
}

// --------------------------------------------------------------- compact
// Merge bins by total community degree.
constexpr int kMergeThreadMax = 16;
constexpr int kMergeWarpMax = 256;   // table kWarpCap
constexpr int kMergeBlockMax = 4096; // table kBlockCap

__global__ void __launch_bounds__(256) k_comm_compact(AggArgs a, int64_t n) {
  const int lane = threadIdx.x & 31;
  unsigned long long md = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = base + threadIdx.x;
    int bin = -1;
    int32_t k = -1;
    if (c < n) {
      const int64_t m0 = a.coff[c], m1 = a.coff[c + 1];
      if (m1 > m0) {
        k = (int32_t)a.newid[c];
        const int64_t h0 = a.hoff[c], h1 = a.hoff[c + 1];
        a.kcoff[k] = m0;
        a.kcnt[k] = (int32_t)(m1 - m0);
        a.obegin[k] = h0;
        a.Knew[k] = a.Sigma[c];
        const int64_t cd = h1 - h0;
        a.oend[k] = h1;  // row capacity until the merge writes the true end
        if (cd > 0) {
          bin = cd <= kMergeThreadMax ? 0 : cd <= kMergeWarpMax ? 1 : cd <= kMergeBlockMax ? 2 : 3;
          if ((unsigned long long)cd > md) md = (unsigned long long)cd;
        }
      }
    }
#pragma unroll
    for (int b = 0; b < kNumBins; ++b) {
      const bool p = bin == b;
      const unsigned mask = __ballot_sync(kFull, p);
      if (!mask) continue;
      const int leader = __ffs(mask) - 1;
      unsigned long long top = 0;
      if (lane == leader) top = atomicAdd(&a.ctr->bin_count[4 + b], (unsigned long long)__popc(mask));
      top = __shfl_sync(kFull, top, leader);
      if (p) a.mbins[b][top + __popc(mask & lanemask_lt())] = k;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long x = __shfl_xor_sync(kFull, md, o);
    md = x > md ? x : md;
  }
  if (lane == 0 && md) atomicMax(&a.ctr->maxdeg, md);
}

__global__ void k_dendro(int32_t *C, const int32_t *Cp, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    C[v] = Cp[C[v]];
}

// --------------------------------------------------------------- merge
__device__ __forceinline__ void tbl_add(int32_t *keys, unsigned long long *vals, uint32_t mask, int32_t key,
                                        long long w, Counters *ctr) {
  uint32_t s = slot_of(key, mask);
  for (uint32_t t = 0; t <= mask; ++t) {
    int32_t k = ((volatile int32_t *)keys)[s];
    if (k == kEmpty) k = atomicCAS(keys + s, kEmpty, key), k = (k == kEmpty) ? key : k;
    if (k == key) {
      atomicAdd(vals + s, (unsigned long long)w);
      return;
    }
    s = (s + 1) & mask;
  }
  atomicOr(&ctr->error, (unsigned long long)ERR_HASH);
}

__device__ __forceinline__ void gtbl_add(int32_t *keys, unsigned long long *vals, uint32_t mask, int32_t key,
                                         long long w, Counters *ctr) {
  uint32_t s = slot_of(key, mask);
  for (uint32_t t = 0; t <= mask; ++t) {
    int32_t k = __ldcg(keys + s);
    if (k == kEmpty) k = atomicCAS(keys + s, kEmpty, key), k = (k == kEmpty) ? key : k;
    if (k == key) {
      atomicAdd(vals + s, (unsigned long long)w);
      return;
    }
    s = (s + 1) & mask;
  }
  atomicOr(&ctr->error, (unsigned long long)ERR_HASH);
}

// Thread per community (total degree <= 16): a short list in shared memory.
template <int WK, int NT>
__global__ void __launch_bounds__(NT) k_merge_thread(AggArgs a) {
  __shared__ int32_t skeys[kMergeThreadMax][NT];
  __shared__ long long svals[kMergeThreadMax][NT];
  const unsigned long long cnt = a.ctr->bin_count[4];
  const int t = threadIdx.x;
  for (unsigned long long idx = (unsigned long long)blockIdx.x * NT + t; idx < cnt;
       idx += (unsigned long long)gridDim.x * NT) {
    const int32_t k = a.mbins[0][idx];
    const int64_t m0 = a.kcoff[k], m1 = m0 + a.kcnt[k];
    int nk = 0;
    for (int64_t mi = m0; mi < m1; ++mi) {
      const int32_t v = a.members[mi];
      for (int64_t e = a.g.begin[v]; e < a.g.end[v]; ++e) {
        const int32_t c = a.Cp[__ldg(a.g.col + e)];
        const long long w = load_w<WK>(a.g.w, e);
        int s = 0;
        while (s < nk && skeys[s][t] != c) ++s;
        if (s == nk) {
          if (nk == kMergeThreadMax) {
            atomicOr(&a.ctr->error, (unsigned long long)ERR_HASH);
            continue;
          }
          skeys[s][t] = c;
          svals[s][t] = 0;
          ++nk;
        }
        svals[s][t] += w;
      }
    }
    const int64_t ob = a.obegin[k];
    for (int s = 0; s < nk; ++s) {
      a.ocol[ob + s] = skeys[s][t];
      a.ow[ob + s] = svals[s][t];
    }
    a.oend[k] = ob + nk;
    atomicAdd(&a.ctr->nnz_out, (unsigned long long)nk);
  }
}

// Warp per community (total degree <= 256): shared table of up to 512 slots.
template <int WK, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_merge_warp(AggArgs a) {
  __shared__ int32_t skeys[WARPS][kWarpCap];
  __shared__ unsigned long long svals[WARPS][kWarpCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t *keys = skeys[warp];
  unsigned long long *vals = svals[warp];
  const unsigned long long cnt = a.ctr->bin_count[5];
  for (unsigned long long idx = (unsigned long long)blockIdx.x * WARPS + warp; idx < cnt;
       idx += (unsigned long long)gridDim.x * WARPS) {
    const int32_t k = a.mbins[1][idx];
    const int64_t m0 = a.kcoff[k], m1 = m0 + a.kcnt[k];
    const int64_t ob = a.obegin[k];
    const uint64_t tot = (uint64_t)(a.oend[k] - ob);  // total member degree
    const uint32_t cap = pow2_at_least(2 * tot);
    const uint32_t mask = cap - 1;
    for (uint32_t s = lane; s < cap; s += 32) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncwarp();
    for (int64_t mi = m0; mi < m1; ++mi) {
      const int32_t v = a.members[mi];
      const int64_t e1 = a.g.end[v];
      for (int64_t e = a.g.begin[v] + lane; e < e1; e += 32)
        tbl_add(keys, vals, mask, a.Cp[__ldg(a.g.col + e)], load_w<WK>(a.g.w, e), a.ctr);
    }
    __syncwarp();
    unsigned long long written = 0;
    for (uint32_t s0 = 0; s0 < cap; s0 += 32) {
      const uint32_t s = s0 + lane;
      const int32_t c = s < cap ? keys[s] : kEmpty;
      const bool occ = c != kEmpty;
      const unsigned m = __ballot_sync(kFull, occ);
      if (occ) {
        const int64_t pos = ob + (int64_t)written + __popc(m & lanemask_lt());
        a.ocol[pos] = c;
        a.ow[pos] = (long long)vals[s];
      }
      written += __popc(m);
    }
    if (lane == 0) {
      a.oend[k] = ob + (int64_t)written;
      atomicAdd(&a.ctr->nnz_out, written);
    }
    __syncwarp();
  }
}

// Block per community (total degree <= 4096): shared table of up to 8192
// slots; warps take members round-robin, lanes stride a member's row.
template <int WK, int NT>
__global__ void __launch_bounds__(NT) k_merge_block(AggArgs a) {
  extern __shared__ unsigned long long dyn[];
  unsigned long long *vals = dyn;
  int32_t *keys = (int32_t *)(dyn + kBlockCap);
  __shared__ unsigned long long s_written;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long cnt = a.ctr->bin_count[6];
  for (unsigned long long idx = blockIdx.x; idx < cnt; idx += gridDim.x) {
    const int32_t k = a.mbins[2][idx];
    const int64_t m0 = a.kcoff[k], m1 = m0 + a.kcnt[k];
    const int64_t ob = a.obegin[k];
    const unsigned long long tot = (unsigned long long)(a.oend[k] - ob);
    if (threadIdx.x == 0) s_written = 0;
    __syncthreads();
    uint64_t distinct = tot < (unsigned long long)a.gamma ? tot : (unsigned long long)a.gamma;
    const uint32_t cap = pow2_at_least(2 * distinct);
    const uint32_t mask = cap - 1;
    for (uint32_t s = threadIdx.x; s < cap; s += NT) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncthreads();
    for (int64_t mi = m0 + warp; mi < m1; mi += NT / 32) {
      const int32_t v = a.members[mi];
      const int64_t e1 = a.g.end[v];
      for (int64_t e = a.g.begin[v] + lane; e < e1; e += 32)
        tbl_add(keys, vals, mask, a.Cp[__ldg(a.g.col + e)], load_w<WK>(a.g.w, e), a.ctr);
    }
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < cap; s += NT) {
      const int32_t c = keys[s];
      if (c == kEmpty) continue;
      const unsigned long long pos = atomicAdd(&s_written, 1ull);
      a.ocol[ob + (int64_t)pos] = c;
      a.ow[ob + (int64_t)pos] = (long long)vals[s];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      a.oend[k] = ob + (int64_t)s_written;
      atomicAdd(&a.ctr->nnz_out, s_written);
    }
    __syncthreads();
  }
}

// Block per community beyond 4096 entries: a global-memory table slice.
// Members with long rows are scanned by the whole block, the rest by warps.
template <int WK, int NT>
__global__ void __launch_bounds__(NT) k_merge_global(AggArgs a) {
  __shared__ unsigned long long s_written;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t *keys = a.ws.keys + (int64_t)blockIdx.x * a.ws.slice;
  unsigned long long *vals = a.ws.vals + (int64_t)blockIdx.x * a.ws.slice;
  const unsigned long long cnt = a.ctr->bin_count[7];
  for (unsigned long long idx = blockIdx.x; idx < cnt; idx += gridDim.x) {
    const int32_t k = a.mbins[3][idx];
    const int64_t m0 = a.kcoff[k], m1 = m0 + a.kcnt[k];
    const int64_t ob = a.obegin[k];
    const unsigned long long tot = (unsigned long long)(a.oend[k] - ob);
    if (threadIdx.x == 0) s_written = 0;
    __syncthreads();
    uint64_t distinct = tot < (unsigned long long)a.gamma ? tot : (unsigned long long)a.gamma;
    const uint32_t cap = pow2_at_least(2 * distinct);
    if ((int64_t)cap > a.ws.slice) {
      if (threadIdx.x == 0) atomicOr(&a.ctr->error, (unsigned long long)ERR_HASH);
      continue;
    }
    const uint32_t mask = cap - 1;
    for (uint32_t s = threadIdx.x; s < cap; s += NT) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncthreads();
    // short member rows: a warp each
    for (int64_t mi = m0 + warp; mi < m1; mi += NT / 32) {
      const int32_t v = a.members[mi];
      const int64_t e0 = a.g.begin[v], e1 = a.g.end[v];
      if (e1 - e0 > 1024) continue;
      for (int64_t e = e0 + lane; e < e1; e += 32)
        gtbl_add(keys, vals, mask, a.Cp[__ldg(a.g.col + e)], load_w<WK>(a.g.w, e), a.ctr);
    }
    // long member rows: the whole block
    for (int64_t mi = m0; mi < m1; ++mi) {
      const int32_t v = a.members[mi];
      const int64_t e0 = a.g.begin[v], e1 = a.g.end[v];
      if (e1 - e0 <= 1024) continue;
      for (int64_t e = e0 + threadIdx.x; e < e1; e += NT)
        gtbl_add(keys, vals, mask, a.Cp[__ldg(a.g.col + e)], load_w<WK>(a.g.w, e), a.ctr);
    }
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < cap; s += NT) {
      const int32_t c = __ldcg(keys + s);
      if (c == kEmpty) continue;
      const unsigned long long pos = atomicAdd(&s_written, 1ull);
      a.ocol[ob + (int64_t)pos] = c;
      a.ow[ob + (int64_t)pos] = (long long)__ldcg(vals + s);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      a.oend[k] = ob + (int64_t)s_written;
      atomicAdd(&a.ctr->nnz_out, s_written);
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------- modularity
// Warp per vertex: internal weight sum_{j in row(i), memb[j] == memb[i]} w_ij
// (self-loop entries included) and, when sigma_out is given, the row sum
// K_i added into sigma_out[memb[i]].
template <int WK>
__global__ void __launch_bounds__(256) k_mod_rows(GView g, const int32_t *memb, int64_t *sigma_out, Counters *ctr) {
  const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
  const int lane = threadIdx.x & 31;
  unsigned long long sin = 0;
  for (int64_t i = warp; i < g.n; i += nw) {
    const int32_t ci = memb[i];
    long long in = 0, k = 0;
    for (int64_t e = g.begin[i] + lane; e < g.end[i]; e += 32) {
      const long long w = load_w<WK>(g.w, e);
      k += w;
      if (memb[__ldg(g.col + e)] == ci) in += w;
    }
    in = warp_sum(in);
    if (sigma_out) {
      k = warp_sum(k);
      if (lane == 0 && k) atomicAdd((unsigned long long *)(sigma_out + ci), as_ull(k));
    }
    sin += (unsigned long long)in;
  }
  if (lane == 0 && sin) atomicAdd(&ctr->q_sin, sin);
}

__global__ void __launch_bounds__(256) k_sigma_sq(const int64_t *sigma, int64_t n, Counters *ctr) {
  unsigned long long lo = 0, hi = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long s = (unsigned long long)sigma[c];
    const unsigned long long sq = s * s;  // Sigma_c <= 2m < 2^32
    lo += sq & 0xFFFFFFFFull;
    hi += sq >> 32;
  }
  lo = warp_sum_u(lo);
  hi = warp_sum_u(hi);
  if ((threadIdx.x & 31) == 0) {
    if (lo) atomicAdd(&ctr->q_tot_lo, lo);
    if (hi) atomicAdd(&ctr->q_tot_hi, hi);
  }
}

__global__ void k_mark_used(const int32_t *x, int64_t n, unsigned long long *used) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    used[x[i]] = 1;
}

__global__ void k_relabel(int32_t *x, int64_t n, const int64_t *newid) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (int32_t)newid[x[i]];
}

template <int WK>
void merge_t(const AggArgs &a, int num_sms, cudaStream_t s) {
  static bool attr_done = false;
  constexpr int kNT = 256;
  constexpr size_t kSmem = (size_t)kBlockCap * (sizeof(unsigned long long) + sizeof(int32_t));
  if (!attr_done) {
    cudaFuncSetAttribute(k_merge_block<WK, kNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    attr_done = true;
  }
  k_merge_thread<WK, 128><<<num_sms * 8, 128, 0, s>>>(a);
  k_merge_warp<WK, 8><<<num_sms * 4, 256, 0, s>>>(a);
  k_merge_block<WK, kNT><<<num_sms * 2, kNT, kSmem, s>>>(a);
  if (a.ws.blocks > 0) k_merge_global<WK, 1024><<<a.ws.blocks, 1024, 0, s>>>(a);
}

template <int WK>
void mod_rows_t(const GView &g, const int32_t *memb, int64_t *sigma_out, Counters *ctr, int num_sms, cudaStream_t s) {
  k_mod_rows<WK><<<grid_for(g.n * 32, 256, num_sms, 16), 256, 0, s>>>(g, memb, sigma_out, ctr);
}

}  // namespace

size_t scan_tmp_elems(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

void scan_u64(const unsigned long long *in, int64_t *out, int64_t n, int mode, long long *tmp,
              unsigned long long *total, cudaStream_t s) {
  if (n <= 0) {
    cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
    return;
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (mode == 0) k_scan_reduce<0><<<(unsigned)nb, kScanNT, 0, s>>>(in, n, tmp);
  else k_scan_reduce<1><<<(unsigned)nb, kScanNT, 0, s>>>(in, n, tmp);
  k_scan_blocks<<<1, kScanNT, 0, s>>>(tmp, nb, total);
  if (mode == 0) k_scan_down<0><<<(unsigned)nb, kScanNT, 0, s>>>(in, out, n, tmp);
  else k_scan_down<1><<<(unsigned)nb, kScanNT, 0, s>>>(in, out, n, tmp);
}

void agg_count_scan(const AggArgs &a, int num_sms, cudaStream_t s) {
  const int64_t n = a.g.n;
  cudaMemsetAsync(a.cnt, 0, (size_t)n * sizeof(unsigned long long), s);
  cudaMemsetAsync(a.cdeg, 0, (size_t)n * sizeof(unsigned long long), s);
  k_comm_count<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(a.g, a.Cp, a.cnt, a.cdeg);
  scan_u64(a.cnt, a.newid, n, 1, a.scan_tmp, &a.ctr->scan_total[0], s);
  scan_u64(a.cnt, a.coff, n, 0, a.scan_tmp, &a.ctr->scan_total[1], s);
  scan_u64(a.cdeg, a.hoff, n, 0, a.scan_tmp, &a.ctr->scan_total[2], s);
  k_write_total<<<1, 1, 0, s>>>(a.newid, n, &a.ctr->scan_total[0]);
  k_write_total<<<1, 1, 0, s>>>(a.coff, n, &a.ctr->scan_total[1]);
  k_write_total<<<1, 1, 0, s>>>(a.hoff, n, &a.ctr->scan_total[2]);
}

void agg_scatter_compact(const AggArgs &a, int num_sms, cudaStream_t s) {
  const int64_t n = a.g.n;
  // cnt is reused as the scatter cursor
  cudaMemsetAsync(a.cnt, 0, (size_t)n * sizeof(unsigned long long), s);
  k_comm_scatter<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(n, a.Cp, a.cnt, a.coff, a.newid, a.members);
  k_comm_compact<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(a, n);
}

void agg_merge(const AggArgs &a, int64_t gamma, int num_sms, cudaStream_t s) {
  if (gamma <= 0) return;
  (void)gamma;
  // a.wkind describes the input G'
  switch (a.wkind) {
    case W_UNIT: merge_t<W_UNIT>(a, num_sms, s); break;
    case W_I32: merge_t<W_I32>(a, num_sms, s); break;
    default: merge_t<W_I64>(a, num_sms, s); break;
  }
}

void dendrogram_lookup(int32_t *C, const int32_t *Cp, int64_t n, int num_sms, cudaStream_t s) {
  if (n <= 0) return;
  k_dendro<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(C, Cp, n);
}

void modularity_sums(const GView &g, int wkind, const int32_t *memb, const int64_t *sigma, int64_t *sigma_scratch,
                     Counters *ctr, int num_sms, cudaStream_t s) {
  if (g.n <= 0) return;
  int64_t *sig_out = nullptr;
  if (!sigma) {
    cudaMemsetAsync(sigma_scratch, 0, (size_t)g.n * sizeof(int64_t), s);
    sig_out = sigma_scratch;
    sigma = sigma_scratch;
  }
  switch (wkind) {
    case W_UNIT: mod_rows_t<W_UNIT>(g, memb, sig_out, ctr, num_sms, s); break;
    case W_I32: mod_rows_t<W_I32>(g, memb, sig_out, ctr, num_sms, s); break;
    default: mod_rows_t<W_I64>(g, memb, sig_out, ctr, num_sms, s); break;
  }
  k_sigma_sq<<<grid_for(g.n, 256, num_sms, 16), 256, 0, s>>>(sigma, g.n, ctr);
}

void renumber_dense(int32_t *x, int64_t n, int64_t idspace, unsigned long long *used, int64_t *newid,
                    long long *tmp, unsigned long long *total, int num_sms, cudaStream_t s) {
  if (n <= 0 || idspace <= 0) {
    cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
    return;
  }
  cudaMemsetAsync(used, 0, (size_t)idspace * sizeof(unsigned long long), s);
  k_mark_used<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(x, n, used);
  scan_u64(used, newid, idspace, 1, tmp, total, s);
  k_relabel<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(x, n, newid);
}

}  // namespace lv
