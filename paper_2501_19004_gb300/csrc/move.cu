// Local-moving phase of the Louvain method on sm_103a (arXiv 2501.19004,
// Sec. 4.2.2 Algorithm 2 and its GPU form Algorithm 5).
//
// One bucket step of the deterministic schedule:
//   k_select   marks the unprocessed vertices of the bucket processed (vertex
//              pruning, Sec. 4.1.6) and sorts them into degree bins;
//   k_move_*   one decision per vertex against the snapshot (C', Sigma'):
//              scanCommunities (Algorithm 2) into a table, the argmax of
//              Eq. 2 scaled by 2m^2, the Pick-Less rejection (Sec. 4.3.1),
//              and, for movers, the exact gain and the re-marking of the
//              neighbours; decisions go to a mover list;
//   hubs       (degree > 32768) are split into chunks over the whole grid
//              (big.cu);
//   k_apply    applies the moves: C'[i] = c*, Sigma' by 64-bit atomics.
// In the asynchronous form (one bucket per iteration) each mover applies its
// own move at the decision instead (emit_move) and k_apply is not launched.
// The paper's per-vertex global hashtables of 2|E| slots (Sec. 4.3.2) become
// register tables (thread bin), shared-memory open addressing (warp and block
// bins) and global tables for hubs only.
#include <climits>

#include <algorithm>
#include <cooperative_groups.h>

#include "internal.h"
#include "learn.cuh"
#include "tables.cuh"

namespace lv {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ------------------------------------------------------------------ select
// Each thread takes 8 consecutive vertices (one 8-byte load of their flags);
// per bin, a warp scan places every thread's selections and one shared
// atomic per warp and one global atomic per block and tile reserve space,
// so a bin list holds each warp's vertices in increasing order.
constexpr int kSelVPT = 8;

__global__ void __launch_bounds__(256) k_select(MoveArgs a) {
  __shared__ unsigned s_cnt[kMoveBins + 1];
  __shared__ unsigned long long s_base[kMoveBins];
  const int64_t n = a.g.n;
  const int lane = threadIdx.x & 31;
  const bool pow2 = (a.nbuckets & (a.nbuckets - 1)) == 0;
  const uint32_t salt = a.iter ? a.iter[0] : a.salt;
  constexpr int64_t kTile = 256 * kSelVPT;
  for (int64_t tile = (int64_t)blockIdx.x * kTile; tile < n; tile += (int64_t)gridDim.x * kTile) {
    if (threadIdx.x <= kMoveBins) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i0 = tile + (int64_t)threadIdx.x * kSelVPT;
    const bool whole = i0 + kSelVPT <= n;
    unsigned long long fl = 0, vbw = 0;
    if (whole) {
      fl = *reinterpret_cast<const unsigned long long *>(a.flag + i0);
      if (fl && a.vbin) vbw = *reinterpret_cast<const unsigned long long *>(a.vbin + i0);
    } else {
#pragma unroll
      for (int v = 0; v < kSelVPT; ++v)
        if (i0 + v < n) {
          fl |= (unsigned long long)a.flag[i0 + v] << (8 * v);
          if (a.vbin) vbw |= (unsigned long long)a.vbin[i0 + v] << (8 * v);
        }
    }
    unsigned long long clear = 0;
    int vb[kSelVPT];
    unsigned cnt[kMoveBins];
#pragma unroll
    for (int b = 0; b < kMoveBins; ++b) cnt[b] = 0;
    unsigned nsel = 0;
#pragma unroll
    for (int v = 0; v < kSelVPT; ++v) {
      const int64_t i = i0 + v;
      vb[v] = -1;
      bool cand = false;
      if (a.learn.record && i < n) {  // the previous bucket's neighbour moves
        const uint32_t mn = a.learn.marks_next[i];
        if (mn) {
          a.learn.marks[i] += mn;
          a.learn.marks_next[i] = 0;
        }
      }
      bool live = ((fl >> (8 * v)) & 0xFFull) != 0;
      uint32_t local = (uint32_t)i;
      if (live && a.batch.gid) {  // batched: only graphs still moving, hashed by their local ids
        const int32_t gg = a.batch.gid[i];
        live = a.batch.moving[gg] != 0;
        local = (uint32_t)(i - a.batch.vo[gg]);
      }
      if (live) {
        const uint32_t h = fmix32(local ^ salt);
        const uint32_t bk = pow2 ? (h & (a.nbuckets - 1)) : (h % a.nbuckets);
        if (bk == a.bucket) {
          if (a.learn.enabled && (a.learn.min_degree == 0 || a.g.end[i] - a.g.begin[i] >= a.learn.min_degree) &&
              a.learn.feat[i].w > 0.f) {
            cand = true;  // the predictor decides (k_mlp_select); the flag stays until then
          } else {
            clear |= 0xFFull << (8 * v);
            ++nsel;
            int b = -1;
            if (a.vbin) {
              const unsigned byte = (unsigned)((vbw >> (8 * v)) & 0xFFull);
              if (byte != 0xFFu) b = (int)byte;
            } else {
              const int64_t deg = a.g.end[i] - a.g.begin[i];
              if (deg > 0) b = move_bin(deg, a.sched.group_max, a.sched.half_max, a.sched.warp_max);
            }
            if (b >= 0) {
              vb[v] = b;
#pragma unroll
              for (int q = 0; q < kMoveBins; ++q) cnt[q] += (q == b) ? 1u : 0u;
            }
          }
        }
      }
      if (a.learn.enabled) {
        const unsigned cmask = __ballot_sync(kFull, cand);
        if (cmask) {
          const int leader = __ffs(cmask) - 1;
          unsigned long long base = 0;
          if (lane == leader) base = atomicAdd(&a.ctr->cand_count, (unsigned long long)__popc(cmask));
          base = __shfl_sync(kFull, base, leader);
          if (cand) a.learn.cand[base + __popc(cmask & lanemask_lt())] = (int32_t)i;
        }
      }
    }
    if (clear) {
      if (whole) {
        *reinterpret_cast<unsigned long long *>(a.flag + i0) = fl & ~clear;
      } else {
#pragma unroll
        for (int v = 0; v < kSelVPT; ++v)
          if ((clear >> (8 * v)) & 0xFFull) a.flag[i0 + v] = 0;
      }
    }
    // per bin: this thread's offset within the warp, the warp's offset
    // within the block
    unsigned woff[kMoveBins], wbase[kMoveBins];
#pragma unroll
    for (int b = 0; b < kMoveBins; ++b) {
      unsigned x = cnt[b];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
      }
      woff[b] = x - cnt[b];
      const unsigned wtot = __shfl_sync(kFull, x, 31);
      unsigned wb = 0;
      if (lane == 0 && wtot) wb = atomicAdd(&s_cnt[b], wtot);
      wbase[b] = __shfl_sync(kFull, wb, 0);
    }
    nsel = warp_sum_u(nsel);
    if (lane == 0 && nsel) atomicAdd(&s_cnt[kMoveBins], (unsigned)nsel);
    __syncthreads();
    if (threadIdx.x < kMoveBins && s_cnt[threadIdx.x])
      s_base[threadIdx.x] = atomicAdd(&a.ctr->bin_count[threadIdx.x], (unsigned long long)s_cnt[threadIdx.x]);
    if (threadIdx.x == kMoveBins && s_cnt[kMoveBins])
      atomicAdd(&a.ctr->it_evaluated, (unsigned long long)s_cnt[kMoveBins]);
    __syncthreads();
#pragma unroll
    for (int b = 0; b < kMoveBins; ++b) {
      if (!cnt[b]) continue;
      unsigned long long pos = s_base[b] + wbase[b] + woff[b];
#pragma unroll
      for (int v = 0; v < kSelVPT; ++v)
        if (vb[v] == b) a.bins[b][pos++] = (int32_t)(i0 + v);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ learned select
// One warp per 16 candidates: features, the BF16 MLP on the tensor cores, and
// the skip decision.  Evaluated vertices are marked processed and binned;
// skipped ones keep their flag for a later iteration.
__global__ void __launch_bounds__(256) k_mlp_select(MoveArgs a) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  MlpFrags f;
  mlp_load_frags(a.learn.params, f, lane);
  const int64_t cnt = (int64_t)a.ctr->cand_count;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long evaluated = 0, skipped = 0;
  for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < cnt; tile += warps) {
    const int64_t r0 = tile * 16 + g, r1 = r0 + 8;
    const int32_t i0 = r0 < cnt ? a.learn.cand[r0] : -1;
    const int32_t i1 = r1 < cnt ? a.learn.cand[r1] : -1;
    float x0[2] = {0.f, 0.f}, x1[2] = {0.f, 0.f};
    float xf[kFeatures];
    if (i0 >= 0) {
      vertex_features(a.g, a.Cp, a.Sigma, a.two_m, a.learn, i0, a.learn.feat[i0], xf);
      x0[0] = xf[2 * t];
      x0[1] = xf[2 * t + 1];
    }
    if (i1 >= 0) {
      vertex_features(a.g, a.Cp, a.Sigma, a.two_m, a.learn, i1, a.learn.feat[i1], xf);
      x1[0] = xf[2 * t];
      x1[1] = xf[2 * t + 1];
    }
    float h1[4][4], h2[4][4], l0, l1;
    mlp_tile_forward(f, x0, x1, h1, h2, l0, l1, t);
    // lane t = 0 of each quad decides row g, lane t = 1 row g + 8
    const int32_t mine = t == 0 ? i0 : (t == 1 ? i1 : -1);
    const float logit = t == 0 ? l0 : l1;
    const bool eval = mine >= 0 && logit >= a.learn.thr_logit;
    int bin = -1;
    if (eval) {
      a.flag[mine] = 0;
      const int64_t deg = a.g.end[mine] - a.g.begin[mine];
      if (deg > 0) bin = move_bin(deg, a.sched.group_max, a.sched.half_max, a.sched.warp_max);
      ++evaluated;
    } else if (mine >= 0) {
      ++skipped;
      if (a.learn.skip_clears) a.flag[mine] = 0;
    }
#pragma unroll
    for (int b = 0; b < kMoveBins; ++b) {
      const unsigned m = __ballot_sync(kFull, bin == b);
      if (!m) continue;
      const int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&a.ctr->bin_count[b], (unsigned long long)__popc(m));
      base = __shfl_sync(kFull, base, leader);
      if (bin == b) a.bins[b][base + __popc(m & lanemask_lt())] = mine;
    }
  }
  evaluated = warp_sum_u(evaluated);
  skipped = warp_sum_u(skipped);
  if (lane == 0) {
    if (evaluated) atomicAdd(&a.ctr->it_evaluated, evaluated);
    if (skipped) atomicAdd(&a.ctr->it_skipped, skipped);
  }
}

// ---------------------------------------------------------------- thread bin
// Degree <= 16: the row lives in registers; K_{i->c} is formed by an all-pairs
// comparison of the (at most 16) neighbour communities.
template <int WK>
__global__ void __launch_bounds__(256) k_move_thread(MoveArgs a) {
  constexpr int D = kThreadMaxDeg;
  const unsigned long long cnt = a.ctr->bin_count[0];
  unsigned long long glo = 0, ghi = 0, gm = 0;
  unsigned long long work[5] = {0, 0, 0, 0, 0};  // vertices, entries, distinct, movers, mover entries
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < cnt;
       base += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long idx = base + threadIdx.x;
    int32_t i = -1, target = -1;
    if (idx < cnt) {
      i = a.bins[0][idx];
      const int64_t b = a.g.begin[i];
      const int deg = (int)(a.g.end[i] - b);
      int32_t jj[D], cc[D];
      uint32_t ww[D];
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
      const long long tm = vertex_two_m(a.batch, a.two_m, i);
      long long Kid = 0;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        if (k >= deg) break;
        Kid += (cc[k] == d) ? ww[k] : 0u;
      }
      long long best_s = LLONG_MIN;
      int32_t best_c = INT_MAX;
      // every community once, at its first occurrence in the row: its weight
      // is the sum over that and the later occurrences (the loops stop at
      // the row's degree)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        if (k >= deg) break;
        const int32_t c = cc[k];
        bool first = (c != kEmpty) && (c != d);
#pragma unroll
        for (int l = 0; l < k; ++l) first = first && (cc[l] != c);
        if (!first) continue;
        long long sum = ww[k];
#pragma unroll
        for (int l = k + 1; l < D; ++l) {
          if (l >= deg) break;
          sum += (cc[l] == c) ? ww[l] : 0u;
        }
        ++work[2];
        const long long s = tm * sum - Ki * a.Sigma[c];
        if (better(s, c, best_s, best_c)) {
          best_s = s;
          best_c = c;
        }
      }
      long long s_d = 0;
      target = finish_decision(tm, a.Sigma, a.iter ? (int)a.iter[1] : a.pickless, d, Ki, Kid, best_s, best_c, glo, ghi, gm, &s_d);
      learn_record(a.learn, a.ctr, a.g, a.Cp, a.Sigma, a.two_m, i, Ki, Kid, best_s, best_c, s_d, target >= 0);
      if (target >= 0) batch_gain(a.batch, i, best_s, s_d);
      work[0] += 1;
      work[1] += (unsigned long long)deg;
      if (target >= 0) {
        work[3] += 1;
        work[4] += (unsigned long long)deg;
#pragma unroll
        for (int k = 0; k < D; ++k)
          if (jj[k] != i) {
            a.flag[jj[k]] = 1;
            learn_mark(a.learn, jj[k]);
          }
      }
    }
    const bool mv = target >= 0;
    const unsigned mask = __ballot_sync(kFull, mv);
    if (mask) {
      const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
      unsigned long long pos = 0;
      if (lane == leader) pos = atomicAdd(&a.ctr->movers, (unsigned long long)__popc(mask));
      pos = __shfl_sync(kFull, pos, leader) + __popc(mask & lanemask_lt());
      if (mv) emit_move(a.async_apply, a.Cp, a.K, a.Sigma, a.mv_vertex, a.mv_target, pos, i, target);
    }
  }
  flush_gains(glo, ghi, gm, a.ctr);
  flush_work(work, a.ctr->mv_work[0]);
}

// Gather kRun entries x, x + stride, ... (< xe) of the row of i that starts
// at b: the community of each neighbour (kEmpty for the self-loop and past
// the end) and the weight.  Consecutive threads read consecutive entries.
template <int WK>
__device__ __forceinline__ void gather_run(const MoveArgs &a, int32_t i, int64_t b, int64_t x, int64_t stride,
                                           int64_t xe, int32_t (&kk)[kRun], uint32_t (&ww)[kRun]) {
#pragma unroll
  for (int u = 0; u < kRun; ++u) {
    kk[u] = -2;
    ww[u] = 0;
    const int64_t p = x + u * stride;
    if (p < xe) {
      kk[u] = __ldg(a.g.col + b + p);
      ww[u] = load_w<WK>(a.g.w, b + p);
    }
  }
#pragma unroll
  for (int u = 0; u < kRun; ++u) kk[u] = (kk[u] >= 0 && kk[u] != i) ? a.Cp[kk[u]] : kEmpty;
}

// ------------------------------------------------------------------ warp bin
// 64 < degree <= 256: one warp, a shared table of up to 512 slots; lanes read
// consecutive entries, up to 8 rounds of 32.
template <int WK, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 4) k_move_warp(MoveArgs a) {
  __shared__ int32_t skeys[WARPS][kWarpCap];
  __shared__ uint32_t svals[WARPS][kWarpCap];
  __shared__ uint16_t socc[WARPS][kWarpMaxDeg];
  __shared__ unsigned snocc[WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t *keys = skeys[warp];
  uint32_t *vals = svals[warp];
  uint16_t *occ = socc[warp];
  unsigned *nocc = &snocc[warp];
  // empty tables; each vertex clears the slots it occupied
  for (int s = lane; s < kWarpCap; s += 32) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  if (lane == 0) *nocc = 0;
  __syncwarp();
  const unsigned long long cnt = a.ctr->bin_count[1];
  unsigned long long glo = 0, ghi = 0, gm = 0;
  unsigned long long work[5] = {0, 0, 0, 0, 0};
  for (unsigned long long idx = (unsigned long long)blockIdx.x * WARPS + warp; idx < cnt;
       idx += (unsigned long long)gridDim.x * WARPS) {
    const int32_t i = a.bins[1][idx];
    const int64_t b = a.g.begin[i], e = a.g.end[i];
    const int64_t deg = e - b;
    const uint32_t mask = kWarpCap - 1;
    for (int64_t x0 = 0; x0 < deg; x0 += 32 * kRun) {
      int32_t kk[kRun];
      uint32_t ww[kRun];
      gather_run<WK>(a, i, b, x0 + lane, 32, deg, kk, ww);
#pragma unroll
      for (int u = 0; u < kRun; ++u)
        if (x0 + u * 32 < deg && kk[u] != kEmpty) sm_insert_list(keys, vals, mask, kk[u], ww[u], occ, nocc, a.ctr);
    }
    __syncwarp();
    const int32_t d = a.Cp[i];
    const long long Ki = a.K[i];
    const long long tm = vertex_two_m(a.batch, a.two_m, i);
    long long best_s = LLONG_MIN, Kid = 0;
    int32_t best_c = INT_MAX;
    const unsigned nk = *(volatile unsigned *)nocc;
    for (unsigned t = lane; t < nk; t += 32) {
      const uint32_t s = occ[t];
      const int32_t c = keys[s];
      const long long v = vals[s];
      keys[s] = kEmpty;
      vals[s] = 0;
      if (c == d) {
        Kid = v;
        continue;
      }
      ++work[2];
      const long long sc = tm * v - Ki * a.Sigma[c];
      if (better(sc, c, best_s, best_c)) {
        best_s = sc;
        best_c = c;
      }
    }
    __syncwarp();
    if (lane == 0) *nocc = 0;
    warp_argmax(best_s, best_c);
    Kid = warp_sum(Kid);
    int32_t target = -1;
    if (lane == 0) {
      long long s_d = 0;
      target = finish_decision(tm, a.Sigma, a.iter ? (int)a.iter[1] : a.pickless, d, Ki, Kid, best_s, best_c, glo, ghi, gm, &s_d);
      learn_record(a.learn, a.ctr, a.g, a.Cp, a.Sigma, a.two_m, i, Ki, Kid, best_s, best_c, s_d, target >= 0);
      if (target >= 0) batch_gain(a.batch, i, best_s, s_d);
      work[0] += 1;
      work[1] += (unsigned long long)deg;
      if (target >= 0) {
        work[3] += 1;
        work[4] += (unsigned long long)deg;
        const unsigned long long pos = atomicAdd(&a.ctr->movers, 1ull);
        emit_move(a.async_apply, a.Cp, a.K, a.Sigma, a.mv_vertex, a.mv_target, pos, i, target);
      }
    }
    target = __shfl_sync(kFull, target, 0);
    if (target >= 0)
      for (int64_t k = b + lane; k < e; k += 32) {
        const int32_t j = __ldg(a.g.col + k);
        if (j != i) {
          a.flag[j] = 1;
          learn_mark(a.learn, j);
        }
      }
    __syncwarp();
  }
  flush_gains(glo, ghi, gm, a.ctr);
  flush_work(work, a.ctr->mv_work[1]);
}

// ----------------------------------------------------------------- group bins
// 16 < degree <= 64 (GS = 8) and 64 < degree <= 128 (GS = 16): GS lanes per
// vertex, 32 / GS vertices per warp, each group with a shared table of up to
// 2 * GS * kRun slots; every lane reads up to kRun entries strided by GS.
// Several vertices per warp keep more independent row and community reads in
// flight than a warp per vertex.
template <int WK, int GS, int WARPS, int BIN>
__global__ void __launch_bounds__(WARPS * 32, 4) k_move_group(MoveArgs a) {
  constexpr int kGroups = 32 / GS;
  constexpr int kSlots = 2 * GS * kRun;
  static_assert(GS * kRun >= (BIN == kGroupBin ? kGroupMaxDeg : kHalfMaxDeg), "a group must hold a whole row");
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
  // the tables start empty and every vertex leaves its table empty: only
  // the occupied slots are visited and cleared
  for (int s = gl; s < kSlots; s += GS) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  if (gl == 0) *nocc = 0;
  __syncwarp();
  const unsigned long long cnt = a.ctr->bin_count[BIN];
  unsigned long long glo = 0, ghi = 0, gm = 0;
  unsigned long long work[5] = {0, 0, 0, 0, 0};
  const unsigned long long stride = (unsigned long long)gridDim.x * WARPS * kGroups;
  for (unsigned long long base = ((unsigned long long)blockIdx.x * WARPS + warp) * kGroups; base < cnt;
       base += stride) {
    const unsigned long long idx = base + grp;
    const bool act = idx < cnt;
    const int32_t i = act ? a.bins[BIN][idx] : 0;
    const int64_t b = act ? a.g.begin[i] : 0;
    const int64_t deg = act ? a.g.end[i] - b : 0;
    const int32_t d = act ? a.Cp[i] : 0;
    const long long Ki = act ? a.K[i] : 0;
    const long long tm = act ? vertex_two_m(a.batch, a.two_m, i) : 0;
    if (act) {
      int32_t kk[kRun];
      uint32_t ww[kRun];
      gather_run<WK>(a, i, b, gl, GS, deg, kk, ww);
#pragma unroll
      for (int u = 0; u < kRun; ++u)
        if (kk[u] != kEmpty) sm_insert_list(keys, vals, kSlots - 1, kk[u], ww[u], occ, nocc, a.ctr);
    }
    __syncwarp();
    const unsigned nk = *(volatile unsigned *)nocc;
    long long best_s = LLONG_MIN, Kid = 0;
    int32_t best_c = INT_MAX;
    for (unsigned t = gl; t < nk; t += GS) {
      const uint32_t s = occ[t];
      const int32_t c = keys[s];
      const long long v = vals[s];
      keys[s] = kEmpty;
      vals[s] = 0;
      if (c == d) {
        Kid = v;
        continue;
      }
      ++work[2];
      const long long sc = tm * v - Ki * a.Sigma[c];
      if (better(sc, c, best_s, best_c)) {
        best_s = sc;
        best_c = c;
      }
    }
    __syncwarp();
    if (gl == 0) *nocc = 0;
    group_argmax<GS>(best_s, best_c);
    Kid = group_sum<GS>(Kid);
    int32_t target = -1;
    if (act && gl == 0) {
      long long s_d = 0;
      target = finish_decision(tm, a.Sigma, a.iter ? (int)a.iter[1] : a.pickless, d, Ki, Kid, best_s, best_c, glo, ghi, gm, &s_d);
      learn_record(a.learn, a.ctr, a.g, a.Cp, a.Sigma, a.two_m, i, Ki, Kid, best_s, best_c, s_d, target >= 0);
      if (target >= 0) batch_gain(a.batch, i, best_s, s_d);
      work[0] += 1;
      work[1] += (unsigned long long)deg;
      if (target >= 0) {
        work[3] += 1;
        work[4] += (unsigned long long)deg;
      }
    }
    // one append per warp for the movers of its groups
    const unsigned mmask = __ballot_sync(kFull, target >= 0);
    if (mmask) {
      const int leader = __ffs(mmask) - 1;
      unsigned long long pos = 0;
      if (lane == leader) pos = atomicAdd(&a.ctr->movers, (unsigned long long)__popc(mmask));
      pos = __shfl_sync(kFull, pos, leader) + __popc(mmask & lanemask_lt());
      if (target >= 0) emit_move(a.async_apply, a.Cp, a.K, a.Sigma, a.mv_vertex, a.mv_target, pos, i, target);
    }
    target = __shfl_sync(kFull, target, grp * GS);
    if (target >= 0)
      for (int64_t k = b + gl; k < b + deg; k += GS) {
        const int32_t j = __ldg(a.g.col + k);
        if (j != i) {
          a.flag[j] = 1;
          learn_mark(a.learn, j);
        }
      }
    __syncwarp();
  }
  flush_gains(glo, ghi, gm, a.ctr);
  flush_work(work, a.ctr->mv_work[BIN]);
}

// ---------------------------------------------------------------- block bins
// 256 < degree <= 1024: 128 threads and a 2048-slot table; 1024 < degree <=
// 4096: 512 threads and an 8192-slot table; 4096 < degree <= 8192: 1024
// threads and a 16384-slot table (dynamic shared memory).  Each thread reads
// 8 entries per round, strided by the block size.
template <int WK, int NT, int CAP, int BIN>
__global__ void __launch_bounds__(NT, NT == 128 ? 8 : NT == 512 ? 2 : 1) k_move_block(MoveArgs a) {
  // dynamic shared memory: keys[CAP], vals[CAP], occupied list[CAP / 2]
  // (a row of degree <= CAP / 2 has at most CAP / 2 distinct keys)
  extern __shared__ uint32_t dyn[];
  int32_t *keys = (int32_t *)dyn;
  uint32_t *vals = dyn + CAP;
  uint16_t *occ = (uint16_t *)(dyn + 2 * CAP);
  __shared__ unsigned s_nocc;
  __shared__ int32_t s_target;
  for (int s = threadIdx.x; s < CAP; s += NT) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  if (threadIdx.x == 0) s_nocc = 0;
  __syncthreads();
  const unsigned long long cnt = a.ctr->bin_count[BIN];
  unsigned long long glo = 0, ghi = 0, gm = 0;
  unsigned long long work[5] = {0, 0, 0, 0, 0};
  for (unsigned long long idx = blockIdx.x; idx < cnt; idx += gridDim.x) {
    const int32_t i = a.bins[BIN][idx];
    const int64_t b = a.g.begin[i], e = a.g.end[i];
    const int64_t deg = e - b;
    for (int64_t x0 = 0; x0 < deg; x0 += (int64_t)NT * kRun) {
      int32_t kk[kRun];
      uint32_t ww[kRun];
      gather_run<WK>(a, i, b, x0 + threadIdx.x, NT, deg, kk, ww);
#pragma unroll
      for (int u = 0; u < kRun; ++u)
        if (kk[u] != kEmpty) sm_insert_list(keys, vals, CAP - 1, kk[u], ww[u], occ, &s_nocc, a.ctr);
    }
    __syncthreads();
    const int32_t d = a.Cp[i];
    const long long Ki = a.K[i];
    const long long tm = vertex_two_m(a.batch, a.two_m, i);
    long long best_s = LLONG_MIN, Kid = 0;
    int32_t best_c = INT_MAX;
    const unsigned nk = s_nocc;
    for (unsigned t = threadIdx.x; t < nk; t += NT) {
      const uint32_t s = occ[t];
      const int32_t c = keys[s];
      const long long v = vals[s];
      keys[s] = kEmpty;
      vals[s] = 0;
      if (c == d) {
        Kid = v;
        continue;
      }
      ++work[2];
      const long long sc = tm * v - Ki * a.Sigma[c];
      if (better(sc, c, best_s, best_c)) {
        best_s = sc;
        best_c = c;
      }
    }
    block_argmax_sum<NT>(best_s, best_c, Kid);
    if (threadIdx.x == 0) {
      long long s_d = 0;
      const int32_t t = finish_decision(tm, a.Sigma, a.iter ? (int)a.iter[1] : a.pickless, d, Ki, Kid, best_s, best_c, glo, ghi, gm, &s_d);
      learn_record(a.learn, a.ctr, a.g, a.Cp, a.Sigma, a.two_m, i, Ki, Kid, best_s, best_c, s_d, t >= 0);
      if (t >= 0) batch_gain(a.batch, i, best_s, s_d);
      work[0] += 1;
      work[1] += (unsigned long long)deg;
      if (t >= 0) {
        work[3] += 1;
        work[4] += (unsigned long long)deg;
        const unsigned long long pos = atomicAdd(&a.ctr->movers, 1ull);
        emit_move(a.async_apply, a.Cp, a.K, a.Sigma, a.mv_vertex, a.mv_target, pos, i, t);
      }
      s_target = t;
      s_nocc = 0;  // every thread read it before block_argmax_sum's barriers
    }
    __syncthreads();
    if (s_target >= 0)
      for (int64_t k = b + threadIdx.x; k < e; k += NT) {
        const int32_t j = __ldg(a.g.col + k);
        if (j != i) {
          a.flag[j] = 1;
          learn_mark(a.learn, j);
        }
      }
    __syncthreads();
  }
  flush_gains(glo, ghi, gm, a.ctr);
  flush_work(work, a.ctr->mv_work[BIN]);
}

// -------------------------------------------------------------- cluster bin
// 8192 < degree <= 32768: a cluster of kClusterSize 1024-thread blocks per
// vertex.  The blocks' shared tables form one table of kClusterSize * 16384
// slots: key k's home slot h lies in block h / 16384, which owns the key and
// probes only within its own 16384 slots.  The row is taken in rounds of
// 8192 entries: every block gathers its share and sends each (key, weight)
// to the owner's staging buffer through distributed shared memory (one
// posted store per entry after one reservation per warp and owner); after a
// cluster barrier every block adds its staged entries into its own part with
// local shared-memory atomics.  Then every block scans the slots it claimed
// for its partial argmax, and block 0 of the cluster reduces the partials and
// decides.  All blocks of a cluster take the same vertices and rounds, so
// they meet the same cluster barriers.
constexpr int kClusterRound = kClusterSize * 1024 * 2;  // entries per round (2 per thread)

__device__ __forceinline__ void owner_insert(int32_t *keys, uint32_t *vals, uint16_t *occ, unsigned *nocc,
                                             uint32_t h, int32_t key, uint32_t w, Counters *ctr) {
  uint32_t s = h % kXlCap;
  for (int t = 0; t < kXlCap; ++t) {
    int32_t cur = ((volatile int32_t *)keys)[s];
    bool claimed = false;
    if (cur == kEmpty) {
      cur = atomicCAS(keys + s, kEmpty, key);
      if (cur == kEmpty) {
        cur = key;
        claimed = true;
      }
    }
    if (cur == key) {
      atomicAdd(vals + s, w);
      if (claimed) occ[atomicAdd(nocc, 1u)] = (uint16_t)s;
      return;
    }
    s = (s + 1) & (kXlCap - 1);
  }
  atomicOr(&ctr->error, (unsigned long long)ERR_HASH);
}

template <int WK>
__global__ void __cluster_dims__(kClusterSize, 1, 1) __launch_bounds__(1024, 1) k_move_cluster(MoveArgs a) {
  namespace cg = cooperative_groups;
  constexpr int NT = 1024;
  constexpr uint32_t kMask = (uint32_t)kClusterSize * kXlCap - 1;
  constexpr int kStage = kClusterRound;  // worst case: a whole round sent to one owner
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int lane = threadIdx.x & 31;
  // dynamic shared memory: keys[16384], vals[16384], occupied list[16384],
  // staged keys[kStage], staged weights[kStage]
  extern __shared__ uint32_t dyn[];
  int32_t *keys = (int32_t *)dyn;
  uint32_t *vals = dyn + kXlCap;
  uint16_t *occ = (uint16_t *)(dyn + 2 * kXlCap);
  int32_t *stage_k = (int32_t *)(dyn + 2 * kXlCap + kXlCap / 2);
  uint32_t *stage_w = (uint32_t *)(stage_k + kStage);
  __shared__ unsigned s_nocc, s_nstage;
  __shared__ long long s_part_s[kClusterSize], s_part_kid[kClusterSize];
  __shared__ int32_t s_part_c[kClusterSize];
  __shared__ int32_t s_target;
  for (int s = threadIdx.x; s < kXlCap; s += NT) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  if (threadIdx.x == 0) {
    s_nocc = 0;
    s_nstage = 0;
  }
  cl.sync();
  const unsigned long long cnt = a.ctr->bin_count[kClusterBin];
  const unsigned long long nclusters = gridDim.x / kClusterSize;
  unsigned long long glo = 0, ghi = 0, gm = 0;
  unsigned long long work[5] = {0, 0, 0, 0, 0};
  for (unsigned long long idx = blockIdx.x / kClusterSize; idx < cnt; idx += nclusters) {
    const int32_t i = a.bins[kClusterBin][idx];
    const int64_t b = a.g.begin[i], e = a.g.end[i];
    const int64_t deg = e - b;
    for (int64_t r0 = 0; r0 < deg; r0 += kClusterRound) {
      // this block's 2 * NT entries of the round, routed to their owners
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int64_t p = r0 + (int64_t)rank * 2 * NT + u * NT + threadIdx.x;
        int32_t key = kEmpty;
        uint32_t w = 0;
        if (p < deg) {
          const int32_t j = __ldg(a.g.col + b + p);
          if (j != i) {
            key = a.Cp[j];
            w = load_w<WK>(a.g.w, b + p);
          }
        }
        const int owner = key == kEmpty ? -1 : (int)(slot_of(key, kMask) / kXlCap);
#pragma unroll
        for (int o = 0; o < kClusterSize; ++o) {
          const unsigned m = __ballot_sync(kFull, owner == o);
          if (!m) continue;
          const int leader = __ffs(m) - 1;
          unsigned base = 0;
          if (lane == leader) base = atomicAdd(cl.map_shared_rank(&s_nstage, o), (unsigned)__popc(m));
          base = __shfl_sync(kFull, base, leader);
          if (owner == o) {
            const unsigned pos = base + __popc(m & lanemask_lt());
            cl.map_shared_rank(stage_k, o)[pos] = key;
            cl.map_shared_rank(stage_w, o)[pos] = w;
          }
        }
      }
      cl.sync();  // every block's staging buffer is complete
      const unsigned ns = s_nstage;
      for (unsigned t = threadIdx.x; t < ns; t += NT) {
        const int32_t key = stage_k[t];
        owner_insert(keys, vals, occ, &s_nocc, slot_of(key, kMask), key, stage_w[t], a.ctr);
      }
      __syncthreads();
      if (threadIdx.x == 0) s_nstage = 0;
      cl.sync();  // staging buffers are free for the next round
    }
    const int32_t d = a.Cp[i];
    const long long Ki = a.K[i];
    const long long tm = vertex_two_m(a.batch, a.two_m, i);
    long long best_s = LLONG_MIN, Kid = 0;
    int32_t best_c = INT_MAX;
    const unsigned nk = s_nocc;
    for (unsigned t = threadIdx.x; t < nk; t += NT) {
      const uint32_t s = occ[t];
      const int32_t c = keys[s];
      const long long v = vals[s];
      keys[s] = kEmpty;
      vals[s] = 0;
      if (c == d) {
        Kid = v;
        continue;
      }
      ++work[2];
      const long long sc = tm * v - Ki * a.Sigma[c];
      if (better(sc, c, best_s, best_c)) {
        best_s = sc;
        best_c = c;
      }
    }
    block_argmax_sum<NT>(best_s, best_c, Kid);
    if (threadIdx.x == 0) {
      s_nocc = 0;  // read by every thread before block_argmax_sum's barriers
      cl.map_shared_rank(s_part_s, 0)[rank] = best_s;
      cl.map_shared_rank(s_part_c, 0)[rank] = best_c;
      cl.map_shared_rank(s_part_kid, 0)[rank] = Kid;
    }
    cl.sync();  // partials in block 0
    if (rank == 0 && threadIdx.x == 0) {
      long long bs = LLONG_MIN, kid = 0;
      int32_t bc = INT_MAX;
      for (int r = 0; r < kClusterSize; ++r) {
        kid += s_part_kid[r];
        if (better(s_part_s[r], s_part_c[r], bs, bc)) {
          bs = s_part_s[r];
          bc = s_part_c[r];
        }
      }
      long long s_d = 0;
      const int32_t t =
          finish_decision(tm, a.Sigma, a.iter ? (int)a.iter[1] : a.pickless, d, Ki, kid, bs, bc, glo, ghi, gm, &s_d);
      learn_record(a.learn, a.ctr, a.g, a.Cp, a.Sigma, a.two_m, i, Ki, kid, bs, bc, s_d, t >= 0);
      if (t >= 0) batch_gain(a.batch, i, bs, s_d);
      work[0] += 1;
      work[1] += (unsigned long long)deg;
      if (t >= 0) {
        work[3] += 1;
        work[4] += (unsigned long long)deg;
        const unsigned long long pos = atomicAdd(&a.ctr->movers, 1ull);
        emit_move(a.async_apply, a.Cp, a.K, a.Sigma, a.mv_vertex, a.mv_target, pos, i, t);
      }
      for (int r = 0; r < kClusterSize; ++r) cl.map_shared_rank(&s_target, r)[0] = t;
    }
    cl.sync();  // decision in every block
    if (s_target >= 0)
      for (int64_t k = b + (int64_t)rank * NT + threadIdx.x; k < e; k += (int64_t)kClusterSize * NT) {
        const int32_t j = __ldg(a.g.col + k);
        if (j != i) {
          a.flag[j] = 1;
          learn_mark(a.learn, j);
        }
      }
  }
  flush_gains(glo, ghi, gm, a.ctr);
  flush_work(work, a.ctr->mv_work[kClusterBin]);
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
// K (row sums on the first pass; given otherwise), Sigma' = K', C' = id,
// all vertices unprocessed; the maximum degree and the size bound of the hub
// tables (sum of pow2(2 min(deg, n')) over degrees > 32768) for the host.
template <int WK>
__global__ void __launch_bounds__(256) k_pass_init(GView g, int first_pass, int64_t *K, int64_t *Sigma,
                                                   int32_t *Cp, uint8_t *flag, Counters *ctr, float4 *feat,
                                                   uint32_t *marks, uint32_t *marks_next, uint8_t *vbin,
                                                   int group_max, int half_max, int warp_max) {
  unsigned long long md = 0, big_slots = 0, big_items = 0;
  const int lane = threadIdx.x & 31;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = g.begin[i], e = g.end[i];
    const unsigned long long deg = (unsigned long long)(e - b);
    if (deg > md) md = deg;
    if (vbin) vbin[i] = deg > 0 ? (uint8_t)move_bin((int64_t)deg, group_max, half_max, warp_max) : (uint8_t)0xFF;
    if (deg > (unsigned long long)kClusterMaxDeg) {  // hubs of the global tables
      big_slots += big_table_cap(deg, (unsigned long long)g.n);
      big_items += 1;
    }
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
    if (feat) {
      feat[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      marks[i] = 0;
      marks_next[i] = 0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long x = __shfl_xor_sync(kFull, md, o);
    md = x > md ? x : md;
  }
  big_slots = warp_sum_u(big_slots);
  big_items = warp_sum_u(big_items);
  if (lane == 0) {
    if (md) atomicMax(&ctr->maxdeg, md);
    if (big_slots) atomicAdd(&ctr->big_slots, big_slots);
    if (big_items) atomicAdd(&ctr->big_items, big_items);
  }
}

__global__ void k_iota(int32_t *x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (int32_t)i;
}

template <int WK>
void move_bucket_t(const MoveArgs &a, const BigArgs &big, int num_sms, cudaStream_t s, KernelProf *prof,
                   const SideStreams *side) {
  static bool attr_done = false;
  constexpr size_t kMidSmem = (size_t)kMidCap * (sizeof(uint32_t) + sizeof(int32_t)) + kMidCap / 2 * sizeof(uint16_t);
  constexpr size_t kBlockSmem =
      (size_t)kBlockCap * (sizeof(uint32_t) + sizeof(int32_t)) + kBlockCap / 2 * sizeof(uint16_t);
  constexpr size_t kXlSmem = (size_t)kXlCap * (sizeof(uint32_t) + sizeof(int32_t)) + kXlCap / 2 * sizeof(uint16_t);
  constexpr size_t kClSmem = (size_t)kXlCap * (sizeof(uint32_t) + sizeof(int32_t) + sizeof(uint16_t)) +
                             (size_t)kClusterRound * (sizeof(int32_t) + sizeof(uint32_t));
  if (!attr_done) {
    cudaFuncSetAttribute(k_move_cluster<WK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClSmem);
    cudaFuncSetAttribute(k_move_block<WK, 512, kBlockCap, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kBlockSmem);
    cudaFuncSetAttribute(k_move_block<WK, 1024, kXlCap, kXlBin>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kXlSmem);
    attr_done = true;
  }
  LV_TIMED(prof, K_SELECT, s, k_select<<<grid_for((a.g.n + kSelVPT - 1) / kSelVPT, 256, num_sms, 8), 256, 0, s>>>(a));
  if (a.learn.enabled) LV_TIMED(prof, K_MLP_SELECT, s, k_mlp_select<<<num_sms * 4, 256, 0, s>>>(a));
  const bool hubs = big.ws.slots > 0;
  if (hubs) big_move_plan(big, s, prof);  // the round count reaches the host while the bins below run
  const int *bk = a.sched.move;
  // the bins' decide kernels are independent (they read the snapshot and
  // append to the mover list with atomics): with `concurrent` they run on
  // side streams at the same time and join before the apply kernel
  const bool conc = side && a.sched.concurrent;
  cudaStream_t s1 = s, s2 = s, s3 = s;
  if (conc) {
    cudaEventRecord(side->fork, s);
    for (int k = 0; k < kSideStreams; ++k) cudaStreamWaitEvent(side->s[k], side->fork, 0);
    s1 = side->s[0];
    s2 = side->s[1];
    s3 = side->s[2];
  }
  LV_TIMED(prof, K_MOVE_THREAD, s1, k_move_thread<WK><<<num_sms * bk[0], 256, 0, s1>>>(a));
  if (a.sched.group_max > kThreadMaxDeg)
    LV_TIMED(prof, K_MOVE_GROUP, s2,
             k_move_group<WK, kGroupLanes, 8, kGroupBin><<<num_sms * bk[kGroupBin], 256, 0, s2>>>(a));
  if (a.sched.half_max > a.sched.group_max)
    LV_TIMED(prof, K_MOVE_HALF, s2,
             k_move_group<WK, kHalfLanes, 8, kHalfBin><<<num_sms * bk[kHalfBin], 256, 0, s2>>>(a));
  LV_TIMED(prof, K_MOVE_WARP, s2, k_move_warp<WK, 8><<<num_sms * bk[1], 256, 0, s2>>>(a));
  LV_TIMED(prof, K_MOVE_MID, s3, k_move_block<WK, 128, kMidCap, 2><<<num_sms * bk[2], 128, kMidSmem, s3>>>(a));
  LV_TIMED(prof, K_MOVE_BLOCK, s3,
           k_move_block<WK, 512, kBlockCap, 3><<<num_sms * bk[3], 512, kBlockSmem, s3>>>(a));
  LV_TIMED(prof, K_MOVE_XL, s,
           k_move_block<WK, 1024, kXlCap, kXlBin><<<num_sms * bk[kXlBin], 1024, kXlSmem, s>>>(a));
  {
    const int clusters = std::max(1, num_sms * bk[kClusterBin] / kClusterSize);
    LV_TIMED(prof, K_MOVE_CLUSTER, s, k_move_cluster<WK><<<clusters * kClusterSize, 1024, kClSmem, s>>>(a));
  }
  if (hubs) big_move_rounds(big, WK, num_sms, s, prof);
  if (conc)
    for (int k = 0; k < kSideStreams; ++k) {
      cudaEventRecord(side->join[k], side->s[k]);
      cudaStreamWaitEvent(s, side->join[k], 0);
    }
  if (!a.async_apply) LV_TIMED(prof, K_APPLY, s, k_apply<<<num_sms * 4, 256, 0, s>>>(a));
}

template <int WK>
void pass_init_t(const GView &g, int first, int64_t *K, int64_t *Sigma, int32_t *Cp, uint8_t *flag, Counters *ctr,
                 int num_sms, cudaStream_t s, const LearnArgs *learn, uint8_t *vbin, const Sched *sched) {
  float4 *feat = (learn && learn->record) ? learn->feat : nullptr;
  uint32_t *marks = (learn && learn->record) ? learn->marks : nullptr;
  uint32_t *marks_next = (learn && learn->record) ? learn->marks_next : nullptr;
  LV_LAUNCH(k_pass_init<WK><<<grid_for(g.n, 256, num_sms, 16), 256, 0, s>>>(g, first, K, Sigma, Cp, flag, ctr, feat,
                                                                             marks, marks_next, vbin,
                                                                             sched ? sched->group_max : 0,
                                                                             sched ? sched->half_max : 0,
                                                                             sched ? sched->warp_max : 0));
}

}  // namespace

void move_bucket(const MoveArgs &a, const BigArgs &big, int wkind, int num_sms, cudaStream_t s, KernelProf *prof,
                 const SideStreams *side) {
  if (a.g.n <= 0) return;
  if (wkind == W_UNIT) move_bucket_t<W_UNIT>(a, big, num_sms, s, prof, side);
  else move_bucket_t<W_U32>(a, big, num_sms, s, prof, side);
}

void pass_init(const GView &g, int wkind, int first_pass, int64_t *K, int64_t *Sigma, int32_t *Cp, uint8_t *flag,
               Counters *ctr, int num_sms, cudaStream_t s, const LearnArgs *learn, uint8_t *vbin, const Sched *sched) {
  if (g.n <= 0) return;
  if (!sched) vbin = nullptr;
  if (wkind == W_UNIT) pass_init_t<W_UNIT>(g, first_pass, K, Sigma, Cp, flag, ctr, num_sms, s, learn, vbin, sched);
  else pass_init_t<W_U32>(g, first_pass, K, Sigma, Cp, flag, ctr, num_sms, s, learn, vbin, sched);
}

void iota_i32(int32_t *x, int64_t n, int num_sms, cudaStream_t s) {
  if (n <= 0) return;
  LV_LAUNCH(k_iota<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(x, n));
}

const char *const kKernelNames[K_NUM_KERNELS] = {
    "select", "move_thread", "move_warp", "move_mid", "move_block", "move_hub", "apply", "pass_init",
    "comm_count", "comm_scatter", "merge_thread", "merge_warp", "merge_mid", "merge_block", "merge_big",
    "dendrogram", "modularity", "renumber", "move_hub_eval", "merge_big_emit", "mlp_select", "move_group", "move_xl", "merge_xl", "move_cluster", "merge_group", "move_half"};

}  // namespace lv
