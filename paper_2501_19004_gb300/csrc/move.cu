// Local-moving phase of the Louvain method on sm_103a (arXiv 2501.19004,
// Sec. 4.2.2 Algorithm 2 and its GPU form Algorithm 5).
//
// One bucket step of the deterministic schedule is four kernels:
//   k_select  marks the unprocessed vertices of the bucket processed (pruning,
//             Sec. 4.1.6) and sorts them into degree bins (warp-aggregated
//             appends);
//   k_move_*  one decision per vertex against the snapshot (C', Sigma'):
//             scanCommunities (Algorithm 2) into a per-vertex table, the
//             argmax of Eq. 2 scaled by 2m^2, the Pick-Less rejection
//             (Sec. 4.3.1), and -- for movers -- the re-marking of the
//             neighbours and the exact gain; decisions go to a mover list;
//   k_apply   applies the moves: C'[i] = c*, Sigma' updates by 64-bit atomics.
// The paper's per-vertex global hashtables of 2|E| slots (Sec. 4.3.2) are
// replaced by register tables (thread bin), shared-memory open addressing
// (warp and block bins) and per-block global slices for hubs only.
#include <climits>

#include "internal.h"

namespace lv {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ void warp_append(bool pred, unsigned long long *counter, int32_t *dst, int32_t v) {
  unsigned mask = __ballot_sync(kFull, pred);
  if (!mask) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
  base = __shfl_sync(kFull, base, leader);
  if (pred) dst[base + __popc(mask & lanemask_lt())] = v;
}

__global__ void __launch_bounds__(256) k_select(MoveArgs a) {
  const int64_t n = a.g.n;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int bin = -1;
    bool sel = false;
    if (i < n && a.flag[i] && fmix32((uint32_t)i ^ a.salt) % a.nbuckets == a.bucket) {
      a.flag[i] = 0;
      sel = true;
      const int64_t deg = a.g.end[i] - a.g.begin[i];
      if (deg > 0) bin = deg <= kThreadMaxDeg ? 0 : deg <= kWarpMaxDeg ? 1 : deg <= kBlockMaxDeg ? 2 : 3;
    }
    unsigned smask = __ballot_sync(kFull, sel);
    if (lane == 0 && smask) atomicAdd(&a.ctr->it_evaluated, (unsigned long long)__popc(smask));
#pragma unroll
    for (int b = 0; b < kNumBins; ++b) warp_append(bin == b, &a.ctr->bin_count[b], a.bins[b], (int32_t)i);
  }
}

// Decision shared by all bins: returns the target or -1.
__device__ __forceinline__ int32_t finish_decision(const MoveArgs &a, int32_t d, long long Ki, long long Kid,
                                                   long long best_s, int32_t best_c, unsigned long long &glo,
                                                   unsigned long long &ghi, unsigned long long &gm) {
  const long long s_d = a.two_m * Kid - Ki * (a.Sigma[d] - Ki);
  if (best_c == INT_MAX || !(best_s > s_d) || (a.pickless && best_c > d)) return -1;
  const unsigned long long gain = (unsigned long long)best_s - (unsigned long long)s_d;
  glo += gain & 0xFFFFFFFFull;
  ghi += gain >> 32;
  gm += 1;
  return best_c;
}

// ---------------------------------------------------------------- thread bin
// Degree <= 16: the row lives in registers; K_{i->c} is formed by an all-pairs
// comparison of the (at most 16) neighbour communities.
template <int WK>
__global__ void __launch_bounds__(256) k_move_thread(MoveArgs a) {
  constexpr int D = kThreadMaxDeg;
  const unsigned long long cnt = a.ctr->bin_count[0];
  unsigned long long glo = 0, ghi = 0, gm = 0;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < cnt;
       base += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long idx = base + threadIdx.x;
    int32_t i = -1, target = -1;
    if (idx < cnt) {
      i = a.bins[0][idx];
      const int64_t b = a.g.begin[i];
      const int deg = (int)(a.g.end[i] - b);
      int32_t jj[D], cc[D];
      long long ww[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        jj[k] = i;
        ww[k] = 0;
        if (k < deg) {
          jj[k] = __ldg(a.g.col + b + k);
          ww[k] = load_w<WK>(a.g.w, b + k);
        }
      }
#pragma unroll
      for (int k = 0; k < D; ++k) cc[k] = (jj[k] == i) ? kEmpty : a.Cp[jj[k]];
      const int32_t d = a.Cp[i];
      const long long Ki = a.K[i];
      long long Kid = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) Kid += (cc[k] == d) ? ww[k] : 0;
      long long best_s = LLONG_MIN;
      int32_t best_c = INT_MAX;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const int32_t c = cc[k];
        bool first = (c != kEmpty) && (c != d);
        long long sum = 0;
#pragma unroll
        for (int l = 0; l < D; ++l) {
          const bool eq = cc[l] == c;
          sum += eq ? ww[l] : 0;
          if (l < k && eq) first = false;
        }
        if (first) {
          const long long s = a.two_m * sum - Ki * a.Sigma[c];
          if (better(s, c, best_s, best_c)) {
            best_s = s;
            best_c = c;
          }
        }
      }
      target = finish_decision(a, d, Ki, Kid, best_s, best_c, glo, ghi, gm);
      if (target >= 0) {
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (jj[k] != i) a.flag[jj[k]] = 1;
      }
    }
    const bool mv = target >= 0;
    unsigned mask = __ballot_sync(kFull, mv);
    if (mask) {
      const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
      unsigned long long pos = 0;
      if (lane == leader) pos = atomicAdd(&a.ctr->movers, (unsigned long long)__popc(mask));
      pos = __shfl_sync(kFull, pos, leader) + __popc(mask & lanemask_lt());
      if (mv) {
        a.mv_vertex[pos] = i;
        a.mv_target[pos] = target;
      }
    }
  }
  flush_gains(glo, ghi, gm, a.ctr);
}

// ------------------------------------------------------ open-addressing tables
// Accumulate (key, w) into a table of mask+1 slots (linear probing).  Tables
// are sized to at least twice the number of distinct keys, so a free slot
// always exists; the probe bound only guards against a sizing bug.
__device__ __forceinline__ void smem_accumulate(int32_t *keys, unsigned long long *vals, uint32_t mask, int32_t key,
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

__device__ __forceinline__ void gmem_accumulate(int32_t *keys, unsigned long long *vals, uint32_t mask, int32_t key,
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

// ------------------------------------------------------------------ warp bin
template <int WK, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_move_warp(MoveArgs a) {
  __shared__ int32_t skeys[WARPS][kWarpCap];
  __shared__ unsigned long long svals[WARPS][kWarpCap];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t *keys = skeys[warp];
  unsigned long long *vals = svals[warp];
  const unsigned long long cnt = a.ctr->bin_count[1];
  unsigned long long glo = 0, ghi = 0, gm = 0;
  for (unsigned long long idx = (unsigned long long)blockIdx.x * WARPS + warp; idx < cnt;
       idx += (unsigned long long)gridDim.x * WARPS) {
    const int32_t i = a.bins[1][idx];
    const int64_t b = a.g.begin[i], e = a.g.end[i];
    const uint32_t cap = pow2_at_least(2 * (uint64_t)(e - b));
    const uint32_t mask = cap - 1;
    for (uint32_t s = lane; s < cap; s += 32) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncwarp();
    for (int64_t k = b + lane; k < e; k += 32) {
      const int32_t j = __ldg(a.g.col + k);
      if (j == i) continue;
      smem_accumulate(keys, vals, mask, a.Cp[j], load_w<WK>(a.g.w, k), a.ctr);
    }
    __syncwarp();
    const int32_t d = a.Cp[i];
    const long long Ki = a.K[i];
    long long best_s = LLONG_MIN, Kid = 0;
    int32_t best_c = INT_MAX;
    for (uint32_t s = lane; s < cap; s += 32) {
      const int32_t c = keys[s];
      if (c == kEmpty) continue;
      const long long v = (long long)vals[s];
      if (c == d) {
        Kid = v;
        continue;
      }
      const long long sc = a.two_m * v - Ki * a.Sigma[c];
      if (better(sc, c, best_s, best_c)) {
        best_s = sc;
        best_c = c;
      }
    }
    warp_argmax(best_s, best_c);
    Kid = warp_sum(Kid);
    int32_t target = -1;
    if (lane == 0) {
      target = finish_decision(a, d, Ki, Kid, best_s, best_c, glo, ghi, gm);
      if (target >= 0) {
        const unsigned long long pos = atomicAdd(&a.ctr->movers, 1ull);
        a.mv_vertex[pos] = i;
        a.mv_target[pos] = target;
      }
    }
    target = __shfl_sync(kFull, target, 0);
    if (target >= 0)
      for (int64_t k = b + lane; k < e; k += 32) {
        const int32_t j = __ldg(a.g.col + k);
        if (j != i) a.flag[j] = 1;
      }
    __syncwarp();
  }
  flush_gains(glo, ghi, gm, a.ctr);
}

// ---------------------------------------------- block reductions (argmax, sum)
template <int NT>
__device__ __forceinline__ void block_argmax_sum(long long &s, int32_t &c, long long &sum) {
  __shared__ long long rs[NT / 32];
  __shared__ int32_t rc[NT / 32];
  __shared__ long long rsum[NT / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  warp_argmax(s, c);
  sum = warp_sum(sum);
  if (lane == 0) {
    rs[warp] = s;
    rc[warp] = c;
    rsum[warp] = sum;
  }
  __syncthreads();
  if (warp == 0) {
    s = lane < NT / 32 ? rs[lane] : LLONG_MIN;
    c = lane < NT / 32 ? rc[lane] : INT_MAX;
    sum = lane < NT / 32 ? rsum[lane] : 0;
    warp_argmax(s, c);
    sum = warp_sum(sum);
  }
  __syncthreads();
}

// ----------------------------------------------------------------- block bin
template <int WK, int NT>
__global__ void __launch_bounds__(NT) k_move_block(MoveArgs a) {
  extern __shared__ unsigned long long dyn[];
  unsigned long long *vals = dyn;
  int32_t *keys = (int32_t *)(dyn + kBlockCap);
  __shared__ int32_t s_target;
  const unsigned long long cnt = a.ctr->bin_count[2];
  unsigned long long glo = 0, ghi = 0, gm = 0;
  for (unsigned long long idx = blockIdx.x; idx < cnt; idx += gridDim.x) {
    const int32_t i = a.bins[2][idx];
    const int64_t b = a.g.begin[i], e = a.g.end[i];
    uint64_t distinct = (uint64_t)(e - b);
    if ((uint64_t)a.g.n < distinct) distinct = (uint64_t)a.g.n;
    const uint32_t cap = pow2_at_least(2 * distinct);
    const uint32_t mask = cap - 1;
    for (uint32_t s = threadIdx.x; s < cap; s += NT) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncthreads();
    for (int64_t k = b + threadIdx.x; k < e; k += NT) {
      const int32_t j = __ldg(a.g.col + k);
      if (j == i) continue;
      smem_accumulate(keys, vals, mask, a.Cp[j], load_w<WK>(a.g.w, k), a.ctr);
    }
    __syncthreads();
    const int32_t d = a.Cp[i];
    const long long Ki = a.K[i];
    long long best_s = LLONG_MIN, Kid = 0;
    int32_t best_c = INT_MAX;
    for (uint32_t s = threadIdx.x; s < cap; s += NT) {
      const int32_t c = keys[s];
      if (c == kEmpty) continue;
      const long long v = (long long)vals[s];
      if (c == d) {
        Kid = v;
        continue;
      }
      const long long sc = a.two_m * v - Ki * a.Sigma[c];
      if (better(sc, c, best_s, best_c)) {
        best_s = sc;
        best_c = c;
      }
    }
    block_argmax_sum<NT>(best_s, best_c, Kid);
    if (threadIdx.x == 0) {
      const int32_t t = finish_decision(a, d, Ki, Kid, best_s, best_c, glo, ghi, gm);
      if (t >= 0) {
        const unsigned long long pos = atomicAdd(&a.ctr->movers, 1ull);
        a.mv_vertex[pos] = i;
        a.mv_target[pos] = t;
      }
      s_target = t;
    }
    __syncthreads();
    if (s_target >= 0)
      for (int64_t k = b + threadIdx.x; k < e; k += NT) {
        const int32_t j = __ldg(a.g.col + k);
        if (j != i) a.flag[j] = 1;
      }
    __syncthreads();
  }
  flush_gains(glo, ghi, gm, a.ctr);
}

// ------------------------------------------------------------------- hub bin
template <int WK, int NT>
__global__ void __launch_bounds__(NT) k_move_hub(MoveArgs a) {
  __shared__ int32_t s_target;
  int32_t *keys = a.ws.keys + (int64_t)blockIdx.x * a.ws.slice;
  unsigned long long *vals = a.ws.vals + (int64_t)blockIdx.x * a.ws.slice;
  const unsigned long long cnt = a.ctr->bin_count[3];
  unsigned long long glo = 0, ghi = 0, gm = 0;
  for (unsigned long long idx = blockIdx.x; idx < cnt; idx += gridDim.x) {
    const int32_t i = a.bins[3][idx];
    const int64_t b = a.g.begin[i], e = a.g.end[i];
    uint64_t distinct = (uint64_t)(e - b);
    if ((uint64_t)a.g.n < distinct) distinct = (uint64_t)a.g.n;
    const uint32_t cap = pow2_at_least(2 * distinct);
    if ((int64_t)cap > a.ws.slice) {  // workspace sized by the host from the max degree
      if (threadIdx.x == 0) atomicOr(&a.ctr->error, (unsigned long long)ERR_HASH);
      continue;
    }
    const uint32_t mask = cap - 1;
    for (uint32_t s = threadIdx.x; s < cap; s += NT) {
      keys[s] = kEmpty;
      vals[s] = 0;
    }
    __syncthreads();
    for (int64_t k = b + threadIdx.x; k < e; k += NT) {
      const int32_t j = __ldg(a.g.col + k);
      if (j == i) continue;
      gmem_accumulate(keys, vals, mask, a.Cp[j], load_w<WK>(a.g.w, k), a.ctr);
    }
    __syncthreads();
    const int32_t d = a.Cp[i];
    const long long Ki = a.K[i];
    long long best_s = LLONG_MIN, Kid = 0;
    int32_t best_c = INT_MAX;
    for (uint32_t s = threadIdx.x; s < cap; s += NT) {
      const int32_t c = __ldcg(keys + s);
      if (c == kEmpty) continue;
      const long long v = (long long)__ldcg(vals + s);
      if (c == d) {
        Kid = v;
        continue;
      }
      const long long sc = a.two_m * v - Ki * a.Sigma[c];
      if (better(sc, c, best_s, best_c)) {
        best_s = sc;
        best_c = c;
      }
    }
    block_argmax_sum<NT>(best_s, best_c, Kid);
    if (threadIdx.x == 0) {
      const int32_t t = finish_decision(a, d, Ki, Kid, best_s, best_c, glo, ghi, gm);
      if (t >= 0) {
        const unsigned long long pos = atomicAdd(&a.ctr->movers, 1ull);
        a.mv_vertex[pos] = i;
        a.mv_target[pos] = t;
      }
      s_target = t;
    }
    __syncthreads();
    if (s_target >= 0)
      for (int64_t k = b + threadIdx.x; k < e; k += NT) {
        const int32_t j = __ldg(a.g.col + k);
        if (j != i) a.flag[j] = 1;
      }
    __syncthreads();
  }
  flush_gains(glo, ghi, gm, a.ctr);
}

// -------------------------------------------------------------------- apply
__global__ void __launch_bounds__(256) k_apply(MoveArgs a) {
  const unsigned long long cnt = a.ctr->movers;
  for (unsigned long long idx = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; idx < cnt;
       idx += (unsigned long long)gridDim.x * blockDim.x) {
    const int32_t i = a.mv_vertex[idx], c = a.mv_target[idx];
    const int32_t d = a.Cp[i];
    const long long Ki = a.K[i];
    a.Cp[i] = c;
    atomicAdd((unsigned long long *)(a.Sigma + d), as_ull(-Ki));
    atomicAdd((unsigned long long *)(a.Sigma + c), as_ull(Ki));
  }
}

// ---------------------------------------------------------------- pass init
template <int WK>
__global__ void __launch_bounds__(256) k_pass_init(GView g, int first_pass, int64_t *K, int64_t *Sigma,
                                                   int32_t *Cp, uint8_t *flag, Counters *ctr) {
  unsigned long long md = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = g.begin[i], e = g.end[i];
    if ((unsigned long long)(e - b) > md) md = (unsigned long long)(e - b);
    long long k;
    if (first_pass) {
      if constexpr (WK == W_UNIT) {
        k = e - b;
      } else {
        k = 0;
        for (int64_t t = b; t < e; ++t) k += load_w<WK>(g.w, t);
      }
      K[i] = k;
    } else {
      k = K[i];
    }
    Sigma[i] = k;
    Cp[i] = (int32_t)i;
    flag[i] = 1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long x = __shfl_xor_sync(kFull, md, o);
    md = x > md ? x : md;
  }
  if ((threadIdx.x & 31) == 0 && md) atomicMax(&ctr->maxdeg, md);
}

__global__ void k_iota(int32_t *x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (int32_t)i;
}

int grid_for(int64_t n, int threads, int num_sms, int per_sm) {
  int64_t g = (n + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

template <int WK>
void move_bucket_t(const MoveArgs &a, int num_sms, cudaStream_t s) {
  static bool attr_done = false;
  constexpr int kBlockNT = 256;
  constexpr size_t kBlockSmem = (size_t)kBlockCap * (sizeof(unsigned long long) + sizeof(int32_t));
  if (!attr_done) {
    cudaFuncSetAttribute(k_move_block<WK, kBlockNT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlockSmem);
    attr_done = true;
  }
  k_select<<<grid_for(a.g.n, 256, num_sms, 16), 256, 0, s>>>(a);
  k_move_thread<WK><<<num_sms * 8, 256, 0, s>>>(a);
  k_move_warp<WK, 8><<<num_sms * 4, 256, 0, s>>>(a);
  k_move_block<WK, kBlockNT><<<num_sms * 2, kBlockNT, kBlockSmem, s>>>(a);
  if (a.ws.blocks > 0) k_move_hub<WK, 1024><<<a.ws.blocks, 1024, 0, s>>>(a);
  k_apply<<<num_sms * 4, 256, 0, s>>>(a);
}

template <int WK>
void pass_init_t(const GView &g, int first, int64_t *K, int64_t *Sigma, int32_t *Cp, uint8_t *flag, Counters *ctr,
                 int num_sms, cudaStream_t s) {
  k_pass_init<WK><<<grid_for(g.n, 256, num_sms, 16), 256, 0, s>>>(g, first, K, Sigma, Cp, flag, ctr);
}

}  // namespace

void move_bucket(const MoveArgs &a, int wkind, int num_sms, cudaStream_t s) {
  if (a.g.n <= 0) return;
  switch (wkind) {
    case W_UNIT: move_bucket_t<W_UNIT>(a, num_sms, s); break;
    case W_I32: move_bucket_t<W_I32>(a, num_sms, s); break;
    default: move_bucket_t<W_I64>(a, num_sms, s); break;
  }
}

void pass_init(const GView &g, int wkind, int first_pass, int64_t *K, int64_t *Sigma, int32_t *Cp, uint8_t *flag,
               Counters *ctr, int num_sms, cudaStream_t s) {
  if (g.n <= 0) return;
  switch (wkind) {
    case W_UNIT: pass_init_t<W_UNIT>(g, first_pass, K, Sigma, Cp, flag, ctr, num_sms, s); break;
    case W_I32: pass_init_t<W_I32>(g, first_pass, K, Sigma, Cp, flag, ctr, num_sms, s); break;
    default: pass_init_t<W_I64>(g, first_pass, K, Sigma, Cp, flag, ctr, num_sms, s); break;
  }
}

void iota_i32(int32_t *x, int64_t n, int num_sms, cudaStream_t s) {
  if (n <= 0) return;
  k_iota<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(x, n);
}

}  // namespace lv
