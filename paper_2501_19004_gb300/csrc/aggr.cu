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
#include "tables.cuh"

namespace lv {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// --------------------------------------------------------------- count
__global__ void __launch_bounds__(256) k_comm_count(GView g, const int32_t *Cp, unsigned long long *cnt,
                                                    unsigned long long *cdeg) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    bool ok = i < g.n;
    const int32_t c = ok ? Cp[i] : -1;
    ok = ok && c >= 0;  // C' < 0: a vertex of a finished graph of a batch
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
    const int32_t c = i < n ? Cp[i] : -1;
    const bool ok = c >= 0;  // C' < 0: a vertex of a finished graph of a batch
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
// Merge bins by total community degree (the degree bins of local moving).
constexpr int kMergeThreadMax = kThreadMaxDeg;

__global__ void __launch_bounds__(256) k_comm_compact(AggArgs a, int64_t n) {
  const int lane = threadIdx.x & 31;
  unsigned long long md = 0, big_slots = 0, big_items = 0;
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
          bin = merge_bin(cd);
          if ((unsigned long long)cd > md) md = (unsigned long long)cd;
          if (bin == kBigBin) {
            big_slots += big_table_cap((unsigned long long)cd, (unsigned long long)a.gamma);
            big_items += 1;
          }
        }
      }
    }
#pragma unroll
    for (int b = 0; b < kMergeBins; ++b) {
      const bool p = bin == b;
      const unsigned mask = __ballot_sync(kFull, p);
      if (!mask) continue;
      const int leader = __ffs(mask) - 1;
      unsigned long long top = 0;
      if (lane == leader) top = atomicAdd(&a.ctr->mbin_count[b], (unsigned long long)__popc(mask));
      top = __shfl_sync(kFull, top, leader);
      if (p) a.mbins[b][top + __popc(mask & lanemask_lt())] = k;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long x = __shfl_xor_sync(kFull, md, o);
    md = x > md ? x : md;
  }
  big_slots = warp_sum_u(big_slots);
  big_items = warp_sum_u(big_items);
  if (lane == 0) {
    if (md) atomicMax(&a.ctr->maxdeg, md);
    if (big_slots) atomicAdd(&a.ctr->big_slots, big_slots);
    if (big_items) atomicAdd(&a.ctr->big_items, big_items);
  }
}

// Degree of every member in community-vertex CSR order (input of the
// member-degree prefix that locates entries of a community's member rows).
// Only the first coff[n] slots hold members (fewer than n when vertices of
// finished graphs of a batch have left); the rest are zero.
__global__ void k_member_deg(GView g, const int32_t *members, const int64_t *coff, unsigned long long *mdeg) {
  const int64_t count = coff[g.n];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < g.n; t += (int64_t)gridDim.x * blockDim.x) {
    if (t >= count) {
      mdeg[t] = 0;
      continue;
    }
    const int32_t v = members[t];
    mdeg[t] = (unsigned long long)(g.end[v] - g.begin[v]);
  }
}

__global__ void k_dendro(int32_t *C, const int32_t *Cp, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = C[v];
    if (x >= 0) C[v] = Cp[x];  // C < 0: frozen (a finished graph of a batch)
  }
}

// --------------------------------------------------------------- merge
// Thread per community (total degree <= 16): a short list in shared memory.
template <int WK, int NT>
__global__ void __launch_bounds__(NT) k_merge_thread(AggArgs a) {
  __shared__ int32_t skeys[kMergeThreadMax][NT];
  __shared__ uint32_t svals[kMergeThreadMax][NT];
  const unsigned long long cnt = a.ctr->mbin_count[0];
  const int t = threadIdx.x;
  unsigned long long work[4] = {0, 0, 0, 0};  // communities, members, entries, written
  for (unsigned long long idx = (unsigned long long)blockIdx.x * NT + t; idx < cnt;
       idx += (unsigned long long)gridDim.x * NT) {
    const int32_t k = a.mbins[0][idx];
    const int64_t m0 = a.kcoff[k], m1 = m0 + a.kcnt[k];
    int nk = 0;
    for (int64_t mi = m0; mi < m1; ++mi) {
      const int32_t v = a.members[mi];
      for (int64_t e = a.g.begin[v]; e < a.g.end[v]; ++e) {
        const int32_t c = a.Cp[__ldg(a.g.col + e)];
        const uint32_t w = load_w<WK>(a.g.w, e);
        ++work[2];
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
    work[0] += 1;
    work[1] += (unsigned long long)(m1 - m0);
    work[3] += (unsigned long long)nk;
  }
  unsigned long long nz[1] = {work[3]};
  flush_work(nz, &a.ctr->nnz_out);
  flush_work(work, a.ctr->mg_work[0]);
}

// Gather run [x, xe) of community k's entry sequence (its members' rows
// concatenated, positions relative to obegin[k]) via the member-degree prefix.
template <int WK>
__device__ __forceinline__ void gather_members(const AggArgs &a, int32_t k, int64_t x, int64_t xe,
                                               int32_t (&kk)[kRun], uint32_t (&ww)[kRun]) {
#pragma unroll
  for (int u = 0; u < kRun; ++u) {
    kk[u] = kEmpty;
    ww[u] = 0;
  }
  if (x >= xe) return;
  const int64_t m0 = a.kcoff[k];
  const int64_t base = a.obegin[k];
  int64_t t = m0 + upper_index(a.mprefix + m0, a.kcnt[k], base + x);
  int64_t mstart = a.mprefix[t];
  int32_t v = a.members[t];
  int64_t rb = a.g.begin[v], rlen = a.g.end[v] - rb;
  int32_t jj[kRun];
#pragma unroll
  for (int u = 0; u < kRun; ++u) {
    jj[u] = -2;
    if (x + u < xe) {
      const int64_t pos = base + x + u;
      while (pos >= mstart + rlen) {
        ++t;
        mstart = a.mprefix[t];
        v = a.members[t];
        rb = a.g.begin[v];
        rlen = a.g.end[v] - rb;
      }
      const int64_t e = rb + (pos - mstart);
      jj[u] = __ldg(a.g.col + e);
      ww[u] = load_w<WK>(a.g.w, e);
    }
  }
#pragma unroll
  for (int u = 0; u < kRun; ++u) kk[u] = jj[u] >= 0 ? a.Cp[jj[u]] : kEmpty;
}

// Group of GS lanes per community (16 < total degree <= 64), 32 / GS
// communities per warp, a 128-slot shared table per group.
template <int WK, int GS, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 4) k_merge_group(AggArgs a) {
  constexpr int kGroups = 32 / GS;
  constexpr int kSlots = 2 * GS * kRun;
  static_assert(GS * kRun >= kGroupMaxDeg, "a group must hold a whole community");
  __shared__ int32_t skeys[WARPS * kGroups][kSlots];
  __shared__ uint32_t svals[WARPS * kGroups][kSlots];
  __shared__ uint16_t socc[WARPS * kGroups][kSlots / 2];
  __shared__ unsigned snocc[WARPS * kGroups];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / GS, gl = lane % GS;
  int32_t *keys = skeys[warp * kGroups + grp];
  uint32_t *vals = svals[warp * kGroups + grp];
  uint16_t *occ = socc[warp * kGroups + grp];
  unsigned *nocc = &snocc[warp * kGroups + grp];
  for (int s = gl; s < kSlots; s += GS) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  if (gl == 0) *nocc = 0;
  __syncwarp();
  const unsigned long long cnt = a.ctr->mbin_count[kMergeGroupBin];
  unsigned long long work[4] = {0, 0, 0, 0};
  const unsigned long long stride = (unsigned long long)gridDim.x * WARPS * kGroups;
  for (unsigned long long base = ((unsigned long long)blockIdx.x * WARPS + warp) * kGroups; base < cnt;
       base += stride) {
    const unsigned long long idx = base + grp;
    const bool act = idx < cnt;
    const int32_t k = act ? a.mbins[kMergeGroupBin][idx] : 0;
    const int64_t ob = act ? a.obegin[k] : 0;
    const int64_t tot = act ? a.oend[k] - ob : 0;  // total member degree
    if (act) {
      int32_t kk[kRun];
      uint32_t ww[kRun];
      const int64_t xs = (int64_t)gl * kRun;
      gather_members<WK>(a, k, xs, xs + kRun < tot ? xs + kRun : tot, kk, ww);
#pragma unroll
      for (int u = 0; u < kRun; ++u)
        if (kk[u] != kEmpty) sm_insert_list(keys, vals, kSlots - 1, kk[u], ww[u], occ, nocc, a.ctr);
    }
    __syncwarp();
    const unsigned nk = *(volatile unsigned *)nocc;
    for (unsigned t = gl; t < nk; t += GS) {
      const uint32_t s = occ[t];
      a.ocol[ob + t] = keys[s];
      a.ow[ob + t] = vals[s];
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncwarp();
    if (act && gl == 0) {
      *nocc = 0;
      a.oend[k] = ob + (int64_t)nk;
      work[0] += 1;
      work[1] += (unsigned long long)a.kcnt[k];
      work[2] += (unsigned long long)tot;
      work[3] += nk;
    }
    __syncwarp();
  }
  unsigned long long nz[1] = {work[3]};
  flush_work(nz, &a.ctr->nnz_out);
  flush_work(work, a.ctr->mg_work[kMergeGroupBin]);
}

// Warp per community (total degree <= 256): shared table of up to 512 slots,
// a run of 8 entries per lane.
template <int WK, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 4) k_merge_warp(AggArgs a) {
  __shared__ int32_t skeys[WARPS][kWarpCap];
  __shared__ uint32_t svals[WARPS][kWarpCap];
  __shared__ uint16_t socc[WARPS][kWarpMaxDeg];
  __shared__ unsigned snocc[WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t *keys = skeys[warp];
  uint32_t *vals = svals[warp];
  uint16_t *occ = socc[warp];
  unsigned *nocc = &snocc[warp];
  // empty tables; each community clears the slots it occupied
  for (int s = lane; s < kWarpCap; s += 32) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  if (lane == 0) *nocc = 0;
  __syncwarp();
  const unsigned long long cnt = a.ctr->mbin_count[1];
  unsigned long long work[4] = {0, 0, 0, 0};
  for (unsigned long long idx = (unsigned long long)blockIdx.x * WARPS + warp; idx < cnt;
       idx += (unsigned long long)gridDim.x * WARPS) {
    const int32_t k = a.mbins[1][idx];
    const int64_t ob = a.obegin[k];
    const int64_t tot = a.oend[k] - ob;  // total member degree
    for (int64_t x0 = 0; x0 < tot; x0 += 32 * kRun) {
      int32_t kk[kRun];
      uint32_t ww[kRun];
      const int64_t xs = x0 + lane * kRun;
      gather_members<WK>(a, k, xs, xs + kRun < tot ? xs + kRun : tot, kk, ww);
#pragma unroll
      for (int u = 0; u < kRun; ++u)
        if (kk[u] != kEmpty) sm_insert_list(keys, vals, kWarpCap - 1, kk[u], ww[u], occ, nocc, a.ctr);
    }
    __syncwarp();
    // the occupied slots are the super-vertex's entries (any order)
    const unsigned nk = *(volatile unsigned *)nocc;
    for (unsigned t = lane; t < nk; t += 32) {
      const uint32_t s = occ[t];
      a.ocol[ob + t] = keys[s];
      a.ow[ob + t] = vals[s];
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncwarp();
    if (lane == 0) {
      *nocc = 0;
      a.oend[k] = ob + (int64_t)nk;
      work[0] += 1;
      work[1] += (unsigned long long)a.kcnt[k];
      work[2] += (unsigned long long)tot;
      work[3] += nk;
    }
    __syncwarp();
  }
  unsigned long long nz[1] = {work[3]};
  flush_work(nz, &a.ctr->nnz_out);
  flush_work(work, a.ctr->mg_work[1]);
}

// Block per community: 128 threads and a 2048-slot table up to 1024
// entries, 512 threads and an 8192-slot table up to 4096, 1024 threads and a
// 16384-slot table up to 8192; a run of 8 consecutive entries per thread.
template <int WK, int NT, int CAP, int BIN>
__global__ void __launch_bounds__(NT, NT == 128 ? 8 : NT == 512 ? 2 : 1) k_merge_block(AggArgs a) {
  // dynamic shared memory: keys[CAP], vals[CAP], occupied list[CAP / 2]
  extern __shared__ uint32_t dyn[];
  int32_t *keys = (int32_t *)dyn;
  uint32_t *vals = dyn + CAP;
  uint16_t *occ = (uint16_t *)(dyn + 2 * CAP);
  __shared__ unsigned s_nocc;
  for (int s = threadIdx.x; s < CAP; s += NT) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  if (threadIdx.x == 0) s_nocc = 0;
  __syncthreads();
  const unsigned long long cnt = a.ctr->mbin_count[BIN];
  unsigned long long work[4] = {0, 0, 0, 0};
  for (unsigned long long idx = blockIdx.x; idx < cnt; idx += gridDim.x) {
    const int32_t k = a.mbins[BIN][idx];
    const int64_t ob = a.obegin[k];
    const int64_t tot = a.oend[k] - ob;
    for (int64_t x0 = 0; x0 < tot; x0 += (int64_t)NT * kRun) {
      int32_t kk[kRun];
      uint32_t ww[kRun];
      const int64_t xs = x0 + (int64_t)threadIdx.x * kRun;
      gather_members<WK>(a, k, xs, xs + kRun < tot ? xs + kRun : tot, kk, ww);
#pragma unroll
      for (int u = 0; u < kRun; ++u)
        if (kk[u] != kEmpty) sm_insert_list(keys, vals, CAP - 1, kk[u], ww[u], occ, &s_nocc, a.ctr);
    }
    __syncthreads();
    const unsigned nk = s_nocc;
    for (unsigned t = threadIdx.x; t < nk; t += NT) {
      const uint32_t s = occ[t];
      a.ocol[ob + t] = keys[s];
      a.ow[ob + t] = vals[s];
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_nocc = 0;
      a.oend[k] = ob + (int64_t)nk;
      work[0] += 1;
      work[1] += (unsigned long long)a.kcnt[k];
      work[2] += (unsigned long long)tot;
      work[3] += nk;
    }
    __syncthreads();
  }
  unsigned long long nz[1] = {work[3]};
  flush_work(nz, &a.ctr->nnz_out);
  flush_work(work, a.ctr->mg_work[BIN]);
}

// --------------------------------------------------------------- modularity
// Internal weight S_in = sum over entries (i, j) with memb[j] == memb[i] of
// w_ij (self-loop entries included) and, when sigma_out is given, the row
// sum K_i added into sigma_out[memb[i]] (Eq. 1's Sigma_c).  Rows are split
// by degree so that no row is walked by too few lanes: rows up to
// kModGroupDeg entries by groups of 8 lanes (4 rows per warp, this kernel),
// rows up to kModWarpDeg by a warp each and longer rows by a 1024-thread
// block each (k_mod_long, from two lists this kernel fills).  A membership
// id outside [0, n) sets ERR_MEMB and its row is skipped (nothing is
// written for it).
constexpr int64_t kModGroupDeg = 64;
constexpr int64_t kModWarpDeg = 4096;

template <int WK>
__global__ void __launch_bounds__(256) k_mod_rows(GView g, const int32_t *memb, int64_t *sigma_out, int32_t *warp_rows,
                                                  int32_t *block_rows, Counters *ctr) {
  constexpr int GS = 8;
  const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / GS;
  const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / GS;
  const int gl = threadIdx.x % GS;
  const int lane = threadIdx.x & 31;
  unsigned long long sin = 0;
  bool bad = false;
  // every lane of a warp runs the same number of rounds (shuffles below)
  const int64_t rounds = (g.n + ngrp - 1) / ngrp;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t i = grp + r * ngrp;
    bool act = i < g.n;
    const int32_t ci = act ? memb[i] : 0;
    if (act && (ci < 0 || ci >= g.n)) {
      bad = true;
      act = false;
    }
    const int64_t rb = act ? g.begin[i] : 0, re = act ? g.end[i] : 0;
    // long rows go to the warp and block lists (one append per warp and list)
    const int cls = (act && re - rb > kModWarpDeg) ? 2 : (act && re - rb > kModGroupDeg) ? 1 : 0;
#pragma unroll
    for (int l = 1; l <= 2; ++l) {
      const unsigned m = __ballot_sync(0xFFFFFFFFu, cls == l && gl == 0);
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(&ctr->mod_count[l - 1], (unsigned long long)__popc(m));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (cls == l && gl == 0) (l == 1 ? warp_rows : block_rows)[base + __popc(m & lanemask_lt())] = (int32_t)i;
      }
    }
    long long in = 0, k = 0;
    if (cls == 0 && act)
      for (int64_t e = rb + gl; e < re; e += GS) {
        const long long w = load_w<WK>(g.w, e);
        k += w;
        if (memb[__ldg(g.col + e)] == ci) in += w;
      }
#pragma unroll
    for (int o = GS / 2; o > 0; o >>= 1) {
      in += __shfl_xor_sync(0xFFFFFFFFu, in, o);
      k += __shfl_xor_sync(0xFFFFFFFFu, k, o);
    }
    if (cls == 0 && act && gl == 0) {
      if (sigma_out && k) atomicAdd((unsigned long long *)(sigma_out + ci), as_ull(k));
      sin += (unsigned long long)in;
    }
  }
  sin = warp_sum_u(sin);
  if ((threadIdx.x & 31) == 0 && sin) atomicAdd(&ctr->q_sin, sin);
  if (bad) atomicOr(&ctr->error, (unsigned long long)ERR_MEMB);
}

// Rows of the warp list (one warp each, 8 entries in flight per lane) and
// of the block list (one 1024-thread block each); the list lengths are in
// ctr->mod_count.  Ids were checked by k_mod_rows.
template <int WK, int NT>
__global__ void __launch_bounds__(NT) k_mod_long(GView g, const int32_t *memb, int64_t *sigma_out,
                                                 const int32_t *rows, const unsigned long long *count, Counters *ctr) {
  constexpr int U = 8;
  constexpr int kRowThreads = NT == 1024 ? 1024 : 32;  // threads per row
  const int64_t cnt = (int64_t)*count;
  const int64_t slot = NT == 1024 ? blockIdx.x : ((int64_t)blockIdx.x * NT + threadIdx.x) / 32;
  const int64_t nslots = NT == 1024 ? gridDim.x : ((int64_t)gridDim.x * NT) / 32;
  const int t = NT == 1024 ? threadIdx.x : (threadIdx.x & 31);
  unsigned long long sin = 0;
  for (int64_t idx = slot; idx < cnt; idx += nslots) {
    const int32_t i = rows[idx];
    const int32_t ci = memb[i];
    const int64_t rb = g.begin[i], re = g.end[i];
    unsigned long long in = 0, k = 0;
    for (int64_t e0 = rb + t; e0 < re; e0 += (int64_t)kRowThreads * U) {
      int32_t jj[U];
      uint32_t ww[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t e = e0 + (int64_t)u * kRowThreads;
        jj[u] = e < re ? __ldg(g.col + e) : -1;
        ww[u] = e < re ? load_w<WK>(g.w, e) : 0u;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        k += ww[u];
        if (jj[u] >= 0 && memb[jj[u]] == ci) in += ww[u];
      }
    }
    sin += in;
    if (sigma_out) {
      k = warp_sum_u(k);
      if ((threadIdx.x & 31) == 0 && k) atomicAdd((unsigned long long *)(sigma_out + ci), k);
    }
  }
  sin = warp_sum_u(sin);
  if ((threadIdx.x & 31) == 0 && sin) atomicAdd(&ctr->q_sin, sin);
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
void merge_t(const AggArgs &a, int num_sms, cudaStream_t s, KernelProf *prof, const SideStreams *side) {
  static bool attr_done = false;
  constexpr size_t kMidSmem = (size_t)kMidCap * (sizeof(uint32_t) + sizeof(int32_t)) + kMidCap / 2 * sizeof(uint16_t);
  constexpr size_t kSmem = (size_t)kBlockCap * (sizeof(uint32_t) + sizeof(int32_t)) + kBlockCap / 2 * sizeof(uint16_t);
  constexpr size_t kXlSmem = (size_t)kXlCap * (sizeof(uint32_t) + sizeof(int32_t)) + kXlCap / 2 * sizeof(uint16_t);
  if (!attr_done) {
    cudaFuncSetAttribute(k_merge_block<WK, 512, kBlockCap, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kSmem);
    cudaFuncSetAttribute(k_merge_block<WK, 1024, kXlCap, kMergeXlBin>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kXlSmem);
    attr_done = true;
  }
  const int *bk = a.sched.merge;
  // the bins write disjoint super-vertex rows: with `concurrent` they run on
  // side streams at the same time and join before returning
  const bool conc = side && a.sched.concurrent;
  cudaStream_t s1 = s, s2 = s, s3 = s;
  if (conc) {
    cudaEventRecord(side->fork, s);
    for (int k = 0; k < kSideStreams; ++k) cudaStreamWaitEvent(side->s[k], side->fork, 0);
    s1 = side->s[0];
    s2 = side->s[1];
    s3 = side->s[2];
  }
  LV_TIMED(prof, K_MERGE_THREAD, s1, k_merge_thread<WK, 128><<<num_sms * bk[0], 128, 0, s1>>>(a));
  LV_TIMED(prof, K_MERGE_GROUP, s1,
           k_merge_group<WK, kGroupLanes, 8><<<num_sms * bk[kMergeGroupBin], 256, 0, s1>>>(a));
  LV_TIMED(prof, K_MERGE_WARP, s2, k_merge_warp<WK, 8><<<num_sms * bk[1], 256, 0, s2>>>(a));
  LV_TIMED(prof, K_MERGE_MID, s3, k_merge_block<WK, 128, kMidCap, 2><<<num_sms * bk[2], 128, kMidSmem, s3>>>(a));
  LV_TIMED(prof, K_MERGE_BLOCK, s3, k_merge_block<WK, 512, kBlockCap, 3><<<num_sms * bk[3], 512, kSmem, s3>>>(a));
  LV_TIMED(prof, K_MERGE_XL, s,
           k_merge_block<WK, 1024, kXlCap, kMergeXlBin><<<num_sms * bk[kMergeXlBin], 1024, kXlSmem, s>>>(a));
  if (a.big.ws.slots > 0) big_merge(a.big, WK, num_sms, s, prof);
  if (conc)
    for (int k = 0; k < kSideStreams; ++k) {
      cudaEventRecord(side->join[k], side->s[k]);
      cudaStreamWaitEvent(s, side->join[k], 0);
    }
}

template <int WK>
void mod_rows_t(const GView &g, const int32_t *memb, int64_t *sigma_out, int32_t *warp_rows, int32_t *block_rows,
                Counters *ctr, int num_sms, cudaStream_t s) {
  cudaMemsetAsync(&ctr->mod_count[0], 0, sizeof(ctr->mod_count), s);
  LV_LAUNCH(k_mod_rows<WK><<<grid_for(g.n * 8, 256, num_sms, 16), 256, 0, s>>>(g, memb, sigma_out, warp_rows,
                                                                                 block_rows, ctr));
  LV_LAUNCH(k_mod_long<WK, 256><<<num_sms * 8, 256, 0, s>>>(g, memb, sigma_out, warp_rows, &ctr->mod_count[0], ctr));
  LV_LAUNCH(k_mod_long<WK, 1024><<<num_sms * 2, 1024, 0, s>>>(g, memb, sigma_out, block_rows, &ctr->mod_count[1],
                                                              ctr));
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
  if (mode == 0) LV_LAUNCH(k_scan_reduce<0><<<(unsigned)nb, kScanNT, 0, s>>>(in, n, tmp));
  else LV_LAUNCH(k_scan_reduce<1><<<(unsigned)nb, kScanNT, 0, s>>>(in, n, tmp));
  LV_LAUNCH(k_scan_blocks<<<1, kScanNT, 0, s>>>(tmp, nb, total));
  if (mode == 0) LV_LAUNCH(k_scan_down<0><<<(unsigned)nb, kScanNT, 0, s>>>(in, out, n, tmp));
  else LV_LAUNCH(k_scan_down<1><<<(unsigned)nb, kScanNT, 0, s>>>(in, out, n, tmp));
}

void agg_count_scan(const AggArgs &a, int num_sms, cudaStream_t s) {
  const int64_t n = a.g.n;
  cudaMemsetAsync(a.cnt, 0, (size_t)n * sizeof(unsigned long long), s);
  cudaMemsetAsync(a.cdeg, 0, (size_t)n * sizeof(unsigned long long), s);
  LV_LAUNCH(k_comm_count<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(a.g, a.Cp, a.cnt, a.cdeg));
  scan_u64(a.cnt, a.newid, n, 1, a.scan_tmp, &a.ctr->scan_total[0], s);
  scan_u64(a.cnt, a.coff, n, 0, a.scan_tmp, &a.ctr->scan_total[1], s);
  scan_u64(a.cdeg, a.hoff, n, 0, a.scan_tmp, &a.ctr->scan_total[2], s);
  LV_LAUNCH(k_write_total<<<1, 1, 0, s>>>(a.newid, n, &a.ctr->scan_total[0]));
  LV_LAUNCH(k_write_total<<<1, 1, 0, s>>>(a.coff, n, &a.ctr->scan_total[1]));
  LV_LAUNCH(k_write_total<<<1, 1, 0, s>>>(a.hoff, n, &a.ctr->scan_total[2]));
}

void agg_scatter_compact(const AggArgs &a, int num_sms, cudaStream_t s) {
  const int64_t n = a.g.n;
  // cnt is reused as the scatter cursor
  cudaMemsetAsync(a.cnt, 0, (size_t)n * sizeof(unsigned long long), s);
  LV_LAUNCH(k_comm_scatter<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(n, a.Cp, a.cnt, a.coff, a.newid, a.members));
  LV_LAUNCH(k_comm_compact<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(a, n));
  // member-degree prefix in community-vertex CSR order (mprefix[t] of the
  // first member of a community equals its row offset hoff)
  LV_LAUNCH(k_member_deg<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(a.g, a.members, a.coff, a.cdeg));
  scan_u64(a.cdeg, a.mprefix, n, 0, a.scan_tmp, &a.ctr->scan_total[3], s);
}

void agg_merge(const AggArgs &a, int64_t gamma, int num_sms, cudaStream_t s, KernelProf *prof,
               const SideStreams *side) {
  if (gamma <= 0) return;
  (void)gamma;
  // a.wkind describes the input G'
  if (a.wkind == W_UNIT) merge_t<W_UNIT>(a, num_sms, s, prof, side);
  else merge_t<W_U32>(a, num_sms, s, prof, side);
}

void dendrogram_lookup(int32_t *C, const int32_t *Cp, int64_t n, int num_sms, cudaStream_t s) {
  if (n <= 0) return;
  LV_LAUNCH(k_dendro<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(C, Cp, n));
}

void modularity_sums(const GView &g, int wkind, const int32_t *memb, const int64_t *sigma, int64_t *sigma_scratch,
                     int32_t *warp_rows, int32_t *block_rows, Counters *ctr, int num_sms, cudaStream_t s) {
  if (g.n <= 0) return;
  int64_t *sig_out = nullptr;
  if (!sigma) {
    cudaMemsetAsync(sigma_scratch, 0, (size_t)g.n * sizeof(int64_t), s);
    sig_out = sigma_scratch;
    sigma = sigma_scratch;
  }
  if (wkind == W_UNIT) mod_rows_t<W_UNIT>(g, memb, sig_out, warp_rows, block_rows, ctr, num_sms, s);
  else mod_rows_t<W_U32>(g, memb, sig_out, warp_rows, block_rows, ctr, num_sms, s);
  LV_LAUNCH(k_sigma_sq<<<grid_for(g.n, 256, num_sms, 16), 256, 0, s>>>(sigma, g.n, ctr));
}

void renumber_dense(int32_t *x, int64_t n, int64_t idspace, unsigned long long *used, int64_t *newid,
                    long long *tmp, unsigned long long *total, int num_sms, cudaStream_t s) {
  if (n <= 0 || idspace <= 0) {
    cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
    return;
  }
  cudaMemsetAsync(used, 0, (size_t)idspace * sizeof(unsigned long long), s);
  LV_LAUNCH(k_mark_used<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(x, n, used));
  scan_u64(used, newid, idspace, 1, tmp, total, s);
  LV_LAUNCH(k_relabel<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(x, n, newid));
}

}  // namespace lv
