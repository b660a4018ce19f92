// The Leiden form (Traag, Waltman and van Eck 2019; the paper's Sec. 5.2 and
// Sec. 6 expect its findings to extend to Leiden): refinement of the
// partition P that local moving produced, and the start of the next pass
// from P.
//
// The refinement is greedy and bucketed (the refine field of
// include/louvain.h).  It reuses the local-moving decision kernels on a
// filtered view of G': every row keeps only its entries inside the
// vertex's community of P (self-loops dropped), written into the spare
// ping-pong buffer at the row's own offsets, so the view is a holey CSR
// with the same row starts.  The decision kernels then run with the refined
// partition (Cr, Sr) in place of (C', Sigma'); their apply step is replaced
// by the two kernels here that let a decision through only when no decision
// of the bucket chose the deciding vertex as its target.
#include <climits>

#include "internal.h"

namespace lv {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kRefineSteps = kRefineChunk / 32;  // 32-entry steps of a chunk's warp: 16

__device__ __forceinline__ bool well_connected(long long two_m, unsigned long long kin, long long Ki, long long Sc) {
  // 2m K_{i->C} >= K_i (Sigma_C - K_i); both sides are below 2^64
  return (unsigned long long)two_m * kin >= (unsigned long long)Ki * (unsigned long long)(Sc - Ki);
}

// Every vertex starts as its own refined community.  A row of at most
// kRefineRowMax entries is filtered by its own lane, four entries' loads in
// flight at a time; a longer row gets one chunk record per kRefineChunk
// entries (taken with one atomic per warp) and k_refine_chunks appends its
// entries.
template <int WK>
__global__ void __launch_bounds__(256) k_refine_rows(RefineArgs r) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < r.g.n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    int64_t b = 0, deg = 0;
    if (v < r.g.n) {
      b = r.g.begin[v];
      deg = r.g.end[v] - b;
      r.Cr[v] = (int32_t)v;
      r.Sr[v] = r.K[v];
    }
    const bool longrow = v < r.g.n && deg > kRefineRowMax;
    const int64_t nch = longrow ? (deg + kRefineChunk - 1) / kRefineChunk : 0;
    if (__ballot_sync(kFull, longrow)) {
      unsigned long long incl = (unsigned long long)nch;  // inclusive scan of the warp's chunk counts
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      unsigned long long c0 = 0;
      if (lane == 31) c0 = atomicAdd(&r.ctr->refine_chunks, incl);
      c0 = __shfl_sync(kFull, c0, 31) + incl - (unsigned long long)nch;
      if (longrow) {
        // the list is sized for the input's rows (louvain_create), so it never runs out
        if ((int64_t)(c0 + nch) > r.chunk_cap) atomicOr(&r.ctr->error, (unsigned long long)ERR_RANGE);
        for (int64_t c = 0; c < nch; ++c)
          if ((int64_t)(c0 + c) < r.chunk_cap) r.chunks[c0 + c] = make_int2((int)v, (int)c);
        r.fend[v] = b;  // the chunks append from here
        r.kin[v] = 0ull;
      }
    }
    if (v < r.g.n && !longrow) {
      const int32_t ci = r.Cp[v];
      int64_t cnt = 0;
      unsigned long long kin = 0;
      for (int64_t k0 = b; k0 < b + deg; k0 += 4) {
        int32_t jj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) jj[u] = k0 + u < b + deg ? __ldg(r.g.col + k0 + u) : -1;
        int32_t cc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cc[u] = (jj[u] >= 0 && jj[u] != (int32_t)v) ? r.Cp[jj[u]] : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (cc[u] == ci) {
            const uint32_t w = load_w<WK>(r.g.w, k0 + u);
            r.fcol[b + cnt] = jj[u];
            if (r.fw) r.fw[b + cnt] = w;
            ++cnt;
            kin += w;
          }
      }
      r.fend[v] = b + cnt;
      const bool ok = well_connected(r.two_m, kin, r.K[v], r.Sigma[ci]);
      r.elig[v] = ok ? 1 : 0;
      r.flag[v] = ok ? kFlagUnproc : 0;
    }
  }
}

// One warp per chunk of a long row: 16 steps of 32 entries with their loads
// in flight, one atomic for the chunk's place in the row, then the writes.
template <int WK>
__global__ void __launch_bounds__(256) k_refine_chunks(RefineArgs r) {
  const int lane = threadIdx.x & 31;
  const unsigned long long total = r.ctr->refine_chunks;
  const long long nch = (long long)total < r.chunk_cap ? (long long)total : r.chunk_cap;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nch; q += nwarps) {
    const int2 rec = r.chunks[q];
    const int32_t i = rec.x;
    const int64_t e = r.g.end[i];
    const int64_t k0 = r.g.begin[i] + (int64_t)rec.y * kRefineChunk;
    const int32_t ci = r.Cp[i];
    int32_t jj[kRefineSteps];
#pragma unroll
    for (int t = 0; t < kRefineSteps; ++t) {
      const int64_t k = k0 + t * 32 + lane;
      jj[t] = k < e ? __ldg(r.g.col + k) : -1;
    }
    unsigned keepbits = 0, n_keep = 0;
    unsigned long long kin = 0;
#pragma unroll
    for (int t = 0; t < kRefineSteps; ++t) {
      const bool keep = jj[t] >= 0 && jj[t] != i && r.Cp[jj[t]] == ci;
      if (keep) {
        keepbits |= 1u << t;
        kin += load_w<WK>(r.g.w, k0 + t * 32 + lane);
      }
      n_keep += __popc(__ballot_sync(kFull, keep));
    }
    unsigned long long at = 0;
    if (lane == 0 && n_keep) at = atomicAdd((unsigned long long *)(r.fend + i), (unsigned long long)n_keep);
    at = __shfl_sync(kFull, at, 0);
#pragma unroll
    for (int t = 0; t < kRefineSteps; ++t) {
      const bool keep = (keepbits >> t) & 1u;
      const unsigned m = __ballot_sync(kFull, keep);
      if (keep) {
        const int64_t pos = (int64_t)at + __popc(m & lanemask_lt());
        r.fcol[pos] = jj[t];
        if (r.fw) r.fw[pos] = load_w<WK>(r.g.w, k0 + t * 32 + lane);
      }
      at += __popc(m);
    }
    kin = warp_sum_u(kin);
    if (lane == 0 && kin) atomicAdd(r.kin + i, kin);
  }
}

// Well-connectedness of the long rows, once their chunks are summed.
__global__ void k_refine_long_elig(RefineArgs r) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < r.g.n; v += (int64_t)gridDim.x * blockDim.x) {
    if (r.g.end[v] - r.g.begin[v] <= kRefineRowMax) continue;
    const bool ok = well_connected(r.two_m, r.kin[v], r.K[v], r.Sigma[r.Cp[v]]);
    r.elig[v] = ok ? 1 : 0;
    r.flag[v] = ok ? kFlagUnproc : 0;
  }
}

// A bucket's decisions: every target a decision chose is marked ...
__global__ void k_refine_choose(const Counters *ctr, const int32_t *mv_target, uint8_t *chosen) {
  const unsigned long long cnt = ctr->movers;
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < cnt;
       k += (unsigned long long)gridDim.x * blockDim.x)
    chosen[mv_target[k]] = 1;
}

// ... and a decision moves its vertex only if no decision chose that vertex
// (so no mover is the target of another, and every refined community keeps
// the id of a member).  The target community is no longer a known singleton.
__global__ void k_refine_apply(const Counters *ctr, const int32_t *mv_vertex, const int32_t *mv_target,
                               const uint8_t *chosen, int32_t *Cr, int64_t *Sr, const int64_t *K, uint32_t *recv) {
  const unsigned long long cnt = ctr->movers;
  for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < cnt;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    const int32_t v = mv_vertex[k];
    if (chosen[v]) continue;
    const int32_t t = mv_target[k];
    const long long Kv = K[v];
    Cr[v] = t;
    atomicAdd((unsigned long long *)(Sr + v), as_ull(-Kv));
    atomicAdd((unsigned long long *)(Sr + t), as_ull(Kv));
    atomicOr(recv + (t >> 5), 1u << (t & 31));
  }
}

// Flags for the rest of the sweep: a vertex still decides if it is well
// connected, no decision has chosen it, and its bucket comes after `bucket`
// (the decision kernels re-mark neighbours of movers; that is undone here).
__global__ void k_refine_flags(int64_t n, const uint8_t *elig, const uint8_t *chosen, uint8_t *flag, uint32_t salt,
                               uint32_t nbuckets, uint32_t bucket) {
  const bool pow2 = (nbuckets & (nbuckets - 1)) == 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t h = fmix32((uint32_t)v ^ salt);
    const uint32_t bk = pow2 ? (h & (nbuckets - 1)) : (h % nbuckets);
    flag[v] = (elig[v] && !chosen[v] && bk > bucket) ? kFlagUnproc : 0;
  }
}

// Start of the next pass from P: super-vertex s of the refined partition
// (dense id Cr[v] of its members v) starts in the community of P of its
// members, represented by the smallest super-vertex of that community.
__global__ void k_fill_i32(int32_t *x, int64_t n, int32_t value) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = value;
}
__global__ void k_leiden_rep(int64_t n, const int32_t *Cp, const int32_t *Cr, int32_t *rep) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    atomicMin(rep + Cp[v], Cr[v]);
}
__global__ void k_leiden_init(int64_t n, const int32_t *Cp, const int32_t *Cr, const int32_t *rep, int32_t *init) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    init[Cr[v]] = rep[Cp[v]];
}

// After pass initialisation (C' = identity, Sigma' = K): every super-vertex
// joins its starting community, whose Sigma' receives its K; a community
// with more than one member is no longer a known singleton.
__global__ void k_leiden_start(int64_t n, const int32_t *init, const int64_t *K, int32_t *Cp, int64_t *Sigma,
                               uint32_t *recv) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = init[s];
    Cp[s] = c;
    if (c == (int32_t)s) continue;
    const long long Ks = K[s];
    atomicAdd((unsigned long long *)(Sigma + c), as_ull(Ks));
    atomicAdd((unsigned long long *)(Sigma + s), as_ull(-Ks));
    atomicOr(recv + (c >> 5), 1u << (c & 31));
  }
}

}  // namespace

void refine_rows(const RefineArgs &r, int wkind, int num_sms, cudaStream_t s) {
  if (r.g.n <= 0) return;
  cudaMemsetAsync(&r.ctr->refine_chunks, 0, sizeof(unsigned long long), s);
  const int grid = grid_for(r.g.n, 256, num_sms, 8);
  if (wkind == W_UNIT) {
    LV_LAUNCH(k_refine_rows<W_UNIT><<<grid, 256, 0, s>>>(r));
    LV_LAUNCH(k_refine_chunks<W_UNIT><<<num_sms * 8, 256, 0, s>>>(r));
  } else {
    LV_LAUNCH(k_refine_rows<W_U32><<<grid, 256, 0, s>>>(r));
    LV_LAUNCH(k_refine_chunks<W_U32><<<num_sms * 8, 256, 0, s>>>(r));
  }
  LV_LAUNCH(k_refine_long_elig<<<grid_for(r.g.n, 256, num_sms, 8), 256, 0, s>>>(r));
}

void refine_resolve(const RefineArgs &r, const int32_t *mv_vertex, const int32_t *mv_target, uint32_t *recv,
                    int num_sms, cudaStream_t s) {
  LV_LAUNCH(k_refine_choose<<<num_sms * 4, 256, 0, s>>>(r.ctr, mv_target, r.chosen));
  LV_LAUNCH(k_refine_apply<<<num_sms * 4, 256, 0, s>>>(r.ctr, mv_vertex, mv_target, r.chosen, r.Cr, r.Sr, r.K, recv));
}

void refine_flags(const RefineArgs &r, uint32_t salt, uint32_t nbuckets, uint32_t bucket, int num_sms, cudaStream_t s) {
  if (r.g.n <= 0) return;
  LV_LAUNCH(k_refine_flags<<<grid_for(r.g.n, 256, num_sms, 8), 256, 0, s>>>(r.g.n, r.elig, r.chosen, r.flag, salt,
                                                                            nbuckets, bucket));
}

void leiden_next_init(int64_t n, const int32_t *Cp, const int32_t *Cr, int32_t *rep, int32_t *init, int num_sms,
                      cudaStream_t s) {
  if (n <= 0) return;
  const int grid = grid_for(n, 256, num_sms, 8);
  LV_LAUNCH(k_fill_i32<<<grid, 256, 0, s>>>(rep, n, INT_MAX));
  LV_LAUNCH(k_leiden_rep<<<grid, 256, 0, s>>>(n, Cp, Cr, rep));
  LV_LAUNCH(k_leiden_init<<<grid, 256, 0, s>>>(n, Cp, Cr, rep, init));
}

void leiden_start(int64_t n, const int32_t *init, const int64_t *K, int32_t *Cp, int64_t *Sigma, uint32_t *recv,
                  int num_sms, cudaStream_t s) {
  if (n <= 0) return;
  LV_LAUNCH(k_leiden_start<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(n, init, K, Cp, Sigma, recv));
}

}  // namespace lv
