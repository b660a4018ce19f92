// Device-side building blocks shared by the Louvain kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lv {

constexpr int32_t kEmpty = -1;          // empty hashtable key
constexpr int kWarp = 32;

// Weight representations of a CSR: unit (no array) or uint32.  The input's
// positive int32 weights are read as uint32; super-vertex graphs store uint32
// too, because every weight is at most 2m < 2^32.
enum WKind : int { W_UNIT = 0, W_U32 = 1 };

template <int WK>
__device__ __forceinline__ uint32_t load_w(const void *w, int64_t e) {
  if constexpr (WK == W_UNIT) {
    return 1u;
  } else {
    return __ldg((const unsigned int *)w + e);
  }
}

// Current graph G' as a "holey" CSR: row i occupies [begin[i], end[i]).
// For a compact CSR end = begin + 1.
struct GView {
  int64_t n;
  const int64_t *begin;
  const int64_t *end;
  const int32_t *col;
  const void *w;
};

// Error bits written by kernels (never a trap).
// ERR_MEMB: a membership id given to the modularity kernel lies outside [0, n).
enum ErrBits : unsigned long long { ERR_HASH = 1ull, ERR_RANGE = 2ull, ERR_TIMEOUT = 4ull, ERR_MEMB = 8ull };

// Small device-resident counters block.
struct Counters {
  unsigned long long bin_count[9];  // local-moving bin sizes of the current bucket (one per move bin)
  unsigned long long movers;        // decisions to move in this bucket
  unsigned long long wide_next;     // work queue of the wide bin: next list position to take
  // ---- zeroed every iteration ----
  unsigned long long it_gain_lo;    // sum of low 32 bits of the gains
  unsigned long long it_gain_hi;    // sum of high 32 bits of the gains
  unsigned long long it_moves;
  unsigned long long it_evaluated;
  unsigned long long it_skipped;    // learned mode: flagged vertices skipped by the predictor
  unsigned long long mv_work[9][5]; // per move bin: vertices, entries, distinct keys, movers, mover entries
  // ---- zeroed every pass ----
  unsigned long long mbin_count[8]; // aggregation bin sizes
  unsigned long long mg_work[7][4]; // per merge bin: communities, members, entries, entries written
  unsigned long long maxdeg;
  unsigned long long big_slots;     // bound on the global table slots of big items
  unsigned long long big_items;     // number of big items (hubs / large communities)
  unsigned long long nnz_out;       // entries written by aggregation
  unsigned long long error;
  unsigned long long q_sin;         // modularity: sum of internal weights
  unsigned long long q_tot_lo;      // modularity: sum of low 32 bits of Sigma_c^2
  unsigned long long q_tot_hi;      // modularity: sum of high 32 bits of Sigma_c^2
  unsigned long long scan_total[4]; // totals of the aggregation scans
  unsigned long long cand_count;    // learned mode: candidates of the bucket for the predictor
  unsigned long long trace_count;   // recorded (features, moved) samples
  unsigned long long mod_count[2];  // modularity: rows handed to warps / to whole blocks
  unsigned long long descents[2];   // validation: adjacent entries with col[k-1] >= col[k] (all / at row starts)
  unsigned long long skip_listed;   // learned mode: vertices the predictor skipped in the current iteration
  unsigned long long sample_blocks; // learned features: neighbour-sample blocks handed out this pass
  unsigned long long sample_chunks; //   and row chunks to sample
  unsigned long long refine_chunks; // Leiden refinement: chunk records of long rows
};
constexpr int kIterCounterWords = 5 + 45;

// MurmurHash3 finaliser (Appleby, public domain).
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

// Salt of the bucket hash for (pass, iteration); see include/louvain.h.
__host__ __device__ __forceinline__ uint32_t bucket_salt(int pass, int iter, uint64_t seed) {
  uint32_t fold = (uint32_t)seed ^ (uint32_t)(seed >> 32);
  uint32_t pt = ((uint32_t)pass << 8) | ((uint32_t)iter & 0xFFu);
  return fmix32(fold ^ (pt * 0x9E3779B1u));
}

// Multiplicative (Fibonacci) hash of a community id into a power-of-two
// table, with one xor-shift so that the low bits see the high ones.
__device__ __forceinline__ uint32_t slot_of(int32_t key, uint32_t mask) {
  uint32_t h = (uint32_t)key * 0x9E3779B1u;
  return (h ^ (h >> 15)) & mask;
}

// Capacity of a big item's global table: twice the keys it can hold (its
// entries, at most the number of possible keys), rounded up to 64 slots.
__host__ __device__ __forceinline__ uint64_t big_table_cap(uint64_t tot, uint64_t keyspace) {
  uint64_t d = tot < keyspace ? tot : keyspace;
  if (d == 0) d = 1;
  return (2 * d + 63) & ~63ull;
}

// Hash of a community id onto [0, cap) for tables of any size
// (multiply-shift range reduction of a mixed 32-bit hash).
__device__ __forceinline__ uint32_t slot_in_range(int32_t key, uint32_t cap) {
  uint32_t h = (uint32_t)key * 0x9E3779B1u;
  h ^= h >> 15;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  return (uint32_t)(((unsigned long long)h * cap) >> 32);
}

// (score, id) pair ordering of the argmax: larger score first, then lower id.
__device__ __forceinline__ bool better(long long s1, int32_t c1, long long s2, int32_t c2) {
  return s1 > s2 || (s1 == s2 && c1 < c2);
}

__device__ __forceinline__ void warp_argmax(long long &s, int32_t &c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long s2 = __shfl_xor_sync(0xFFFFFFFFu, s, o);
    int32_t c2 = __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (better(s2, c2, s, c)) { s = s2; c = c2; }
  }
}

// Argmax and sum over aligned groups of W lanes (W a power of two <= 32).
template <int W>
__device__ __forceinline__ void group_argmax(long long &s, int32_t &c) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    long long s2 = __shfl_xor_sync(0xFFFFFFFFu, s, o);
    int32_t c2 = __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (better(s2, c2, s, c)) { s = s2; c = c2; }
  }
}

template <int W>
__device__ __forceinline__ long long group_sum(long long v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ unsigned long long as_ull(long long v) { return (unsigned long long)v; }

// A decision to move vertex i to community c.  Deterministic schedule: onto
// the mover list at pos, applied by k_apply after all decisions of the
// bucket.  Asynchronous form: applied at once (C'[i], then Sigma' of the old
// and the new community by 64-bit atomics), so that decisions made later in
// the same sweep see it.  A vertex is decided once per sweep, so no other
// thread writes C'[i] meanwhile.
__device__ __forceinline__ void emit_move(int async_apply, int32_t *Cp, const int64_t *K, int64_t *Sigma,
                                          int32_t *mv_vertex, int32_t *mv_target, unsigned long long pos,
                                          int32_t i, int32_t c) {
  if (async_apply) {
    const int32_t d = Cp[i];
    const long long Ki = K[i];
    Cp[i] = c;
    atomicAdd((unsigned long long *)(Sigma + d), as_ull(-Ki));
    atomicAdd((unsigned long long *)(Sigma + c), as_ull(Ki));
  } else {
    mv_vertex[pos] = i;
    mv_target[pos] = c;
  }
}

// Exact accumulation of non-negative 64-bit gains into two 64-bit sums
// (low and high 32-bit halves), reduced per warp before the global atomics.
__device__ __forceinline__ void flush_gains(unsigned long long lo, unsigned long long hi,
                                            unsigned long long moves, Counters *ctr) {
  lo = warp_sum_u(lo);
  hi = warp_sum_u(hi);
  moves = warp_sum_u(moves);
  if ((threadIdx.x & 31) == 0 && (lo | hi | moves)) {
    atomicAdd(&ctr->it_gain_lo, lo);
    atomicAdd(&ctr->it_gain_hi, hi);
    atomicAdd(&ctr->it_moves, moves);
  }
}

// Work counters of one kernel: reduced per warp, then one atomic per field.
template <int N>
__device__ __forceinline__ void flush_work(unsigned long long (&w)[N], unsigned long long *dst) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const unsigned long long v = warp_sum_u(w[k]);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst + k, v);
  }
}

// The decision of Algorithm 5 for vertex i in community d, given the best
// neighbour community (best_s, best_c) and K_{i->d}: returns the target or -1.
// A move needs a strictly larger score than staying and, in Pick-Less mode,
// a target id below d.  The gain s(c*) - s(d) is positive and below 2^64.
__device__ __forceinline__ int32_t finish_decision(long long two_m, const int64_t *Sigma, int pickless, int32_t d,
                                                   long long Ki, long long Kid, long long best_s, int32_t best_c,
                                                   unsigned long long &glo, unsigned long long &ghi,
                                                   unsigned long long &gm, long long *s_d_out = nullptr) {
  const long long s_d = two_m * Kid - Ki * (Sigma[d] - Ki);
  if (s_d_out) *s_d_out = s_d;
  if (best_c == 0x7FFFFFFF || !(best_s > s_d) || (pickless && best_c > d)) return -1;
  const unsigned long long gain = (unsigned long long)best_s - (unsigned long long)s_d;
  glo += gain & 0xFFFFFFFFull;
  ghi += gain >> 32;
  gm += 1;
  return best_c;
}

// Block-wide argmax (score, then lowest id) and sum; the result is valid in
// every thread of warp 0.
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
    s = lane < NT / 32 ? rs[lane] : (long long)0x8000000000000000ull;
    c = lane < NT / 32 ? rc[lane] : 0x7FFFFFFF;
    sum = lane < NT / 32 ? rsum[lane] : 0;
    warp_argmax(s, c);
    sum = warp_sum(sum);
  }
  __syncthreads();
}

// Round up to a power of two (x >= 1).
__host__ __device__ __forceinline__ uint32_t pow2_at_least(uint64_t x) {
  uint32_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace lv
