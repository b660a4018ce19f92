// Open-addressing tables (community id -> summed weight) used by the
// local-moving and aggregation kernels.  Keys are int32 community ids
// (kEmpty = free), values are uint32: every sum that lands in a table is at
// most 2m < 2^32 (a K_{i->c} is bounded by K_i, a super-edge weight by 2m).
// Tables always hold at least twice as many slots as distinct keys, so
// linear probing always finds a slot; the probe bound only guards against a
// sizing error and raises ERR_HASH (the "failed" result of Algorithm 7).
#pragma once
#include "common.cuh"

namespace lv {

// Longest probe sequence of one insert: the paper's MAX_RETRIES of Algorithm
// 7, after which the insert fails (ERR_HASH, LOUVAIN_E_HASH_OVERFLOW).  The
// tables here are sized so that no input reaches it, so the product build
// has no bound but the table size; a build with -DLOUVAIN_MAX_PROBES=k makes
// inserts give up after k probes, which the tests use to exercise the
// failure path.  (A bound read from memory in these loops slowed the hub
// accumulation several times over, so it is a compile-time constant.)
#ifndef LOUVAIN_MAX_PROBES
#define LOUVAIN_MAX_PROBES 0xFFFFFFFFu
#endif
constexpr uint32_t kMaxProbes = LOUVAIN_MAX_PROBES;

constexpr int kRun = 8;  // consecutive entries handled by one thread per round

__device__ __forceinline__ void sm_insert(int32_t *keys, uint32_t *vals, uint32_t mask, int32_t key, uint32_t w,
                                          Counters *ctr) {
  uint32_t s = slot_of(key, mask);
  const uint32_t lim = mask < kMaxProbes ? mask + 1 : kMaxProbes;  // probes allowed
  for (uint32_t t = 0; t < lim; ++t) {
    int32_t k = ((volatile int32_t *)keys)[s];
    if (k == kEmpty) {
      k = atomicCAS(keys + s, kEmpty, key);
      if (k == kEmpty) k = key;
    }
    if (k == key) {
      atomicAdd(vals + s, w);
      return;
    }
    s = (s + 1) & mask;
  }
  atomicOr(&ctr->error, (unsigned long long)ERR_HASH);
}

// sm_insert that also appends a slot it claims for a new key to the table's
// occupied list (occ, *nocc), so that readers visit and clear only the
// occupied slots.
__device__ __forceinline__ void sm_insert_list(int32_t *keys, uint32_t *vals, uint32_t mask, int32_t key, uint32_t w,
                                               uint16_t *occ, unsigned *nocc, Counters *ctr) {
  uint32_t s = slot_of(key, mask);
  const uint32_t lim = mask < kMaxProbes ? mask + 1 : kMaxProbes;  // probes allowed
  for (uint32_t t = 0; t < lim; ++t) {
    int32_t k = ((volatile int32_t *)keys)[s];
    bool claimed = false;
    if (k == kEmpty) {
      k = atomicCAS(keys + s, kEmpty, key);
      if (k == kEmpty) {
        k = key;
        claimed = true;
      }
    }
    if (k == key) {
      atomicAdd(vals + s, w);
      if (claimed) occ[atomicAdd(nocc, 1u)] = (uint16_t)s;
      return;
    }
    s = (s + 1) & mask;
  }
  atomicOr(&ctr->error, (unsigned long long)ERR_HASH);
}

// Global tables of big items use packed 64-bit slots: (key + 1) in the high
// half, the summed weight in the low half (sums stay below 2^32, so adding a
// weight never carries into the key); 0 is an empty slot.  An insert touches
// one word: a CAS claims an empty slot with the first weight, later weights
// of the same key are one 64-bit add.
__device__ __forceinline__ int32_t packed_key(unsigned long long v) { return (int32_t)(uint32_t)(v >> 32) - 1; }
__device__ __forceinline__ uint32_t packed_val(unsigned long long v) { return (uint32_t)v; }

// Insert of (key, w) starting at slot s, whose current content `cur` the
// caller has read: claim an empty slot with a CAS, add to the key's slot, or
// probe on.  Returns the slot it claimed for the key, -1 when the key was
// present.
__device__ __forceinline__ int64_t gm_insert_packed_from(unsigned long long *tab, uint32_t cap, uint32_t s,
                                                         unsigned long long cur, int32_t key, uint32_t w,
                                                         Counters *ctr) {
  const unsigned long long hk = (unsigned long long)(uint32_t)(key + 1) << 32;
  const uint32_t lim = cap < kMaxProbes ? cap : kMaxProbes;  // probes allowed
  for (uint32_t t = 0; t < lim; ++t) {
    if (cur == 0ull) {
      cur = atomicCAS(tab + s, 0ull, hk | w);
      if (cur == 0ull) return (int64_t)s;
    }
    if ((cur & 0xFFFFFFFF00000000ull) == hk) {
      atomicAdd(tab + s, (unsigned long long)w);
      return -1;
    }
    s = (s + 1 == cap) ? 0u : s + 1;
    cur = __ldcg(tab + s);
  }
  atomicOr(&ctr->error, (unsigned long long)ERR_HASH);
  return -1;
}

__device__ __forceinline__ unsigned long long packed_pair(int32_t key, uint32_t w) {
  return ((unsigned long long)(uint32_t)(key + 1) << 32) | w;
}

// Warp-cooperative insert into a shared table: all 32 lanes call it (key =
// kEmpty for nothing).  When the warp holds few distinct keys (a hot
// community), lanes with equal keys are summed first and one lane inserts;
// otherwise every lane inserts its own pair.
__device__ __forceinline__ void warp_insert_sm(int32_t *keys, uint32_t *vals, uint32_t mask, int32_t key, uint32_t w,
                                               Counters *ctr) {
  const unsigned full = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(full, key);
  const bool lead = lane == __ffs(peers) - 1;
  const unsigned leaders = __ballot_sync(full, lead && key != kEmpty);
  if (__popc(leaders) <= 4) {
    unsigned todo = leaders;
    while (todo) {
      const int src = __ffs(todo) - 1;
      todo &= todo - 1;
      const int32_t k0 = __shfl_sync(full, key, src);
      const uint32_t sum = __reduce_add_sync(full, key == k0 ? w : 0u);
      if (lane == src) sm_insert(keys, vals, mask, k0, sum, ctr);
    }
  } else if (key != kEmpty) {
    sm_insert(keys, vals, mask, key, w, ctr);
  }
}

// Block-level exclusive scan of one int64 per thread (NT threads); returns
// the exclusive prefix and the block total in *total.  Uses `scratch`
// (NT/32 + 1 words of shared memory).
template <int NT>
__device__ __forceinline__ long long block_scan_ex(long long v, long long *scratch, long long *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long s = lane < NT / 32 ? scratch[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xFFFFFFFFu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NT / 32) scratch[lane] = s;
  }
  __syncthreads();
  const long long before = warp ? scratch[warp - 1] : 0;
  *total = scratch[NT / 32 - 1];
  __syncthreads();
  return before + x - v;
}

// Largest index k in [0, n) with a[k] <= x (a non-decreasing, a[0] <= x).
__device__ __forceinline__ int64_t upper_index(const int64_t *a, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;  // invariant: a[lo] <= x, answer in [lo, hi)
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

}  // namespace lv
