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
      if ((fl & kFlagUnproc8) && a.vbin)
        vbw = *reinterpret_cast<const unsigned long long *>(a.vbin + i0);
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
      const unsigned vbyte = (unsigned)((vbw >> (8 * v)) & 0xFFull);
      const bool tracked = a.learn.min_degree == 0 ||
                           (a.vbin ? (vbyte & kVbinTracked) != 0
                                   : (i < n && a.g.end[i] - a.g.begin[i] >= a.learn.min_degree));
      bool live = ((fl >> (8 * v)) & (unsigned long long)kFlagUnproc) != 0;
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
          if (a.learn.enabled && tracked && a.learn.feat[i].w > 0.f) {
            cand = true;  // the predictor decides (k_mlp_select); the flag stays until then
          } else {
            clear |= (unsigned long long)kFlagUnproc << (8 * v);
            ++nsel;
            int b = -1;
            if (a.vbin) {
              const unsigned byte = vbyte & kVbinBinMask;
              if (byte != kVbinNone) b = (int)byte;
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
          if ((clear >> (8 * v)) & 0xFFull) a.flag[i0 + v] &= (uint8_t)~kFlagUnproc;
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

// ------------------------------------------------------------ list select
// Completion step of a learned iteration: every vertex of sel_list is
// evaluated (its flag cleared) and sorted into its degree bin.
__global__ void __launch_bounds__(256) k_select_list(MoveArgs a) {
  const int lane = threadIdx.x & 31;
  const unsigned long long cnt = *a.sel_count;
  unsigned long long evaluated = 0;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x; base < cnt;
       base += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long idx = base + threadIdx.x;
    int bin = -1;
    int32_t i = -1;
    if (idx < cnt) {
      i = a.sel_list[idx];
      a.flag[i] &= (uint8_t)~kFlagUnproc;
      ++evaluated;
      if (a.vbin) {
        const unsigned byte = a.vbin[i] & kVbinBinMask;
        if (byte != kVbinNone) bin = (int)byte;
      } else {
        const int64_t deg = a.g.end[i] - a.g.begin[i];
        if (deg > 0) bin = move_bin(deg, a.sched.group_max, a.sched.half_max, a.sched.warp_max);
      }
    }
#pragma unroll
    for (int b = 0; b < kMoveBins; ++b) {
      const unsigned m = __ballot_sync(kFull, bin == b);
      if (!m) continue;
      const int leader = __ffs(m) - 1;
      unsigned long long pos = 0;
      if (lane == leader) pos = atomicAdd(&a.ctr->bin_count[b], (unsigned long long)__popc(m));
      pos = __shfl_sync(kFull, pos, leader);
      if (bin == b) a.bins[b][pos + __popc(m & lanemask_lt())] = i;
    }
  }
  evaluated = warp_sum_u(evaluated);
  if (lane == 0 && evaluated) atomicAdd(&a.ctr->it_evaluated, evaluated);
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
      a.flag[mine] &= (uint8_t)~kFlagUnproc;
      const int64_t deg = a.g.end[mine] - a.g.begin[mine];
      if (deg > 0) bin = move_bin(deg, a.sched.group_max, a.sched.half_max, a.sched.warp_max);
      ++evaluated;
    } else if (mine >= 0) {
      ++skipped;
      if (a.learn.skip_clears) a.flag[mine] &= (uint8_t)~kFlagUnproc;
    }
    if (a.learn.skip_list) {  // the iteration's skipped vertices, for its completion step
      const bool sk = mine >= 0 && !eval;
      const unsigned m = __ballot_sync(kFull, sk);
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(&a.ctr->skip_listed, (unsigned long long)__popc(m));
        base = __shfl_sync(kFull, base, leader);
        if (sk) a.learn.skip_list[base + __popc(m & lanemask_lt())] = mine;
      }
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
          if (jj[k] != i) a.flag[jj[k]] = kFlagUnproc;
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
      mark_neighbours(a.flag, a.g.col, b, e, lane, 32, i);
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
      mark_neighbours(a.flag, a.g.col, b, b + deg, gl, GS, i);
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
      mark_neighbours(a.flag, a.g.col, b, e, threadIdx.x, NT, i);
    __syncthreads();
  }
  flush_gains(glo, ghi, gm, a.ctr);
  flush_work(work, a.ctr->mv_work[BIN]);
}

// ----------------------------------------------------------------- wide bin
// 4096 < degree <= 32768: one 1024-thread block per vertex, one block per
// SM taking vertices from a work queue.  An entry whose neighbour j is alone
// in its community (a known singleton: C'[j] = j and no vertex has moved into
// community j this pass) contributes K_{i->j} = w_ij by itself when rows hold
// no repeated column, so its score is formed at once and kept in a
// per-thread running argmax; such a community is never the vertex's own
// (that would hold i and j).  Only the other entries go through the
// 16384-slot shared table (claims appended to the occupied list once per
// warp); once it holds kWideCap keys, the remaining entries go to
// the block's own global table of kWideSpill packed 64-bit slots (twice the
// largest row, so at most half full), the shared table is flushed into it,
// and the vertex is decided from that table, which its scan leaves empty.
// At iteration 0 of a pass every community is a singleton, so those scans
// touch no table at all.
constexpr int kWideOcc = kWideCap + 1024;  // occupied-list entries: the cap plus one late claim per thread
constexpr int kWideRun = 4;  // entries per thread per round (1024 x 4 in flight per block)

__device__ __forceinline__ bool recv_bit(const uint32_t *recv, int32_t c) {
  return (__ldg(recv + (c >> 5)) >> (c & 31)) & 1u;
}

// Insert into the shared wide table by the whole warp (every lane calls it;
// key = kEmpty for nothing).  Returns false, inserting nothing, once the
// table holds kWideCap keys (*over is set): the caller spills the pair.  The
// count read before a claim lags by at most one claim per thread, so the
// table holds fewer than kWideCap + 1024 keys, at most 13/16 full, and
// probing always finds a slot.  Claimed slots are appended to the occupied
// list with one atomic per warp.
__device__ __forceinline__ bool wide_insert_warp(int32_t *keys, uint32_t *vals, uint16_t *occ, unsigned *nocc,
                                                 int *over, int32_t key, uint32_t w, Counters *ctr) {
  constexpr uint32_t mask = kXlCap - 1;
  int32_t claimed = -1;
  bool ok = true;
  if (key != kEmpty) {
    if (*(volatile int *)over || *(volatile unsigned *)nocc >= (unsigned)kWideCap) {
      *(volatile int *)over = 1;
      ok = false;
    } else {
      uint32_t s = slot_of(key, mask);
      const uint32_t lim = mask < kMaxProbes ? mask + 1 : kMaxProbes;  // probes allowed
      uint32_t t = 0;
      for (; t < lim; ++t) {
        int32_t k = ((volatile int32_t *)keys)[s];
        if (k == kEmpty) {
          k = atomicCAS(keys + s, kEmpty, key);
          if (k == kEmpty) {
            k = key;
            claimed = (int32_t)s;
          }
        }
        if (k == key) {
          atomicAdd(vals + s, w);
          break;
        }
        s = (s + 1) & mask;
      }
      if (t == lim) atomicOr(&ctr->error, (unsigned long long)ERR_HASH);
    }
  }
  const unsigned m = __ballot_sync(kFull, claimed >= 0);
  if (m) {
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(nocc, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (claimed >= 0) occ[base + __popc(m & lanemask_lt())] = (uint16_t)claimed;
  }
  return ok;
}

__device__ __forceinline__ void spill_insert(unsigned long long *tab, int32_t key, uint32_t w, Counters *ctr) {
  const uint32_t home = slot_of(key, kWideSpill - 1);
  gm_insert_packed_from(tab, kWideSpill, home, __ldcg(tab + home), key, w, ctr);
}

template <int WK>
__global__ void __launch_bounds__(1024, 1) k_move_wide(MoveArgs a) {
  constexpr int NT = 1024;
  // dynamic shared memory: keys[16384], vals[16384], occupied list[kWideOcc]
  extern __shared__ uint32_t dyn[];
  int32_t *keys = (int32_t *)dyn;
  uint32_t *vals = dyn + kXlCap;
  uint16_t *occ = (uint16_t *)(dyn + 2 * kXlCap);
  __shared__ unsigned s_nocc;
  __shared__ int s_over;
  __shared__ int32_t s_target;
  __shared__ unsigned long long s_idx;
  unsigned long long *spill = a.wide_spill + (size_t)blockIdx.x * kWideSpill;  // left empty between vertices
  for (int s = threadIdx.x; s < kXlCap; s += NT) {
    keys[s] = kEmpty;
    vals[s] = 0;
  }
  if (threadIdx.x == 0) {
    s_nocc = 0;
    s_over = 0;
  }
  const unsigned long long cnt = a.ctr->bin_count[kXlBin];
  unsigned long long glo = 0, ghi = 0, gm = 0;
  unsigned long long work[5] = {0, 0, 0, 0, 0};
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_idx = atomicAdd(&a.ctr->wide_next, 1ull);
    __syncthreads();
    const unsigned long long idx = s_idx;
    if (idx >= cnt) break;
    const int32_t i = a.bins[kXlBin][idx];
    const int64_t b = a.g.begin[i], e = a.g.end[i];
    const int64_t deg = e - b;
    const long long Ki = a.K[i];
    const long long tm = vertex_two_m(a.batch, a.two_m, i);
    long long best_s = LLONG_MIN, Kid = 0;
    int32_t best_c = INT_MAX;
    for (int64_t x0 = 0; x0 < deg; x0 += (int64_t)NT * kWideRun) {
      int32_t jj[kWideRun], kk[kWideRun];
      uint32_t ww[kWideRun];
#pragma unroll
      for (int u = 0; u < kWideRun; ++u) {
        const int64_t p = x0 + threadIdx.x + (int64_t)u * NT;
        jj[u] = -2;
        ww[u] = 0;
        if (p < deg) {
          jj[u] = __ldg(a.g.col + b + p);
          ww[u] = load_w<WK>(a.g.w, b + p);
        }
      }
#pragma unroll
      for (int u = 0; u < kWideRun; ++u) kk[u] = (jj[u] >= 0 && jj[u] != i) ? a.Cp[jj[u]] : kEmpty;
      bool solo[kWideRun];
#pragma unroll
      for (int u = 0; u < kWideRun; ++u) solo[u] = a.solo && kk[u] != kEmpty && kk[u] == jj[u] && !recv_bit(a.recv, kk[u]);
      long long sig[kWideRun];
#pragma unroll
      for (int u = 0; u < kWideRun; ++u) sig[u] = solo[u] ? a.Sigma[kk[u]] : 0;
#pragma unroll
      for (int u = 0; u < kWideRun; ++u) {
        if (kk[u] == kEmpty) continue;
        if (solo[u]) {
          ++work[2];
          const long long sc = tm * (long long)ww[u] - Ki * sig[u];
          if (better(sc, kk[u], best_s, best_c)) {
            best_s = sc;
            best_c = kk[u];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kWideRun; ++u) {
        const int32_t key = (kk[u] != kEmpty && !solo[u]) ? kk[u] : kEmpty;
        if (!wide_insert_warp(keys, vals, occ, &s_nocc, &s_over, key, ww[u], a.ctr))
          spill_insert(spill, key, ww[u], a.ctr);
      }
    }
    __syncthreads();
    const unsigned nk = s_nocc;
    const bool over = s_over != 0;
    const int32_t d = a.Cp[i];
    if (over) {
      // the shared table's keys join the spilled ones; the vertex is decided
      // from the block's global table, whose slots are cleared as read
      for (unsigned t = threadIdx.x; t < nk; t += NT) {
        const uint16_t sl = occ[t];
        spill_insert(spill, keys[sl], vals[sl], a.ctr);
        keys[sl] = kEmpty;
        vals[sl] = 0;
      }
      __syncthreads();
      for (int r = threadIdx.x; r < kWideSpill; r += NT) {
        const unsigned long long pv = __ldcg(spill + r);
        if (pv == 0ull) continue;
        spill[r] = 0ull;
        const int32_t c = packed_key(pv);
        const long long v = packed_val(pv);
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
    } else {
      for (unsigned t = threadIdx.x; t < nk; t += NT) {
        const uint16_t sl = occ[t];
        const int32_t c = keys[sl];
        const long long v = vals[sl];
        keys[sl] = kEmpty;
        vals[sl] = 0;
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
    }
    block_argmax_sum<NT>(best_s, best_c, Kid);
    if (threadIdx.x == 0) {
      long long s_d = 0;
      const int32_t t = finish_decision(tm, a.Sigma, a.iter ? (int)a.iter[1] : a.pickless, d, Ki, Kid, best_s,
                                        best_c, glo, ghi, gm, &s_d);
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
      s_over = 0;
    }
    __syncthreads();
    if (s_target >= 0)
      mark_neighbours(a.flag, a.g.col, b, e, threadIdx.x, NT, i);
  }
  flush_gains(glo, ghi, gm, a.ctr);
  flush_work(work, a.ctr->mv_work[kXlBin]);
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
    if (a.recv) atomicOr(a.recv + (c >> 5), 1u << (c & 31));  // community c is no longer a known singleton
    if (a.learn.moved_at) a.learn.moved_at[i] = a.learn.stamp;
    atomicAdd((unsigned long long *)(a.Sigma + d), as_ull(-Ki));
    atomicAdd((unsigned long long *)(a.Sigma + c), as_ull(Ki));
  }
}

// --------------------------------------------------- neighbour samples
// Per pass, for the learned feature x7 (see learn.cuh).  The plan kernel
// gives every tracked vertex with a row longer than kSample a sample block
// and one chunk record per kSampleChunk entries of its row (sample_at = -1
// for the others); the chunk kernel then tests the entries of one chunk per
// block and appends the neighbours that pass the pair-hash test to the
// block.  The stored set is fixed by the graph; only its order varies.
__global__ void __launch_bounds__(256) k_sample_plan(GView g, LearnArgs L, Counters *ctr) {
  const int64_t dmin = L.min_degree > kSample ? L.min_degree : kSample + 1;
  const int lane = threadIdx.x & 31;
  // whole warps step together, so the blocks and chunks of a warp's
  // vertices are taken with one atomic each
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = base + threadIdx.x;
    const int64_t deg = v < g.n ? g.end[v] - g.begin[v] : 0;
    const bool mine = v < g.n && deg >= dmin;
    const int64_t nch = mine ? (deg + kSampleChunk - 1) / kSampleChunk : 0;
    const unsigned m = __ballot_sync(kFull, mine);
    if (!m) {
      if (v < g.n) L.sample_at[v] = -1;
      continue;
    }
    unsigned long long incl = (unsigned long long)nch;  // inclusive scan of the chunk counts
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    const unsigned long long wtot = __shfl_sync(kFull, incl, 31);
    unsigned long long b0 = 0, cb = 0;
    if (lane == 0) {
      b0 = atomicAdd(&ctr->sample_blocks, (unsigned long long)__popc(m));
      cb = atomicAdd(&ctr->sample_chunks, wtot);
    }
    b0 = __shfl_sync(kFull, b0, 0);
    cb = __shfl_sync(kFull, cb, 0);
    if (v >= g.n) continue;
    int32_t at = -1;
    if (mine) {
      const unsigned long long blk = b0 + __popc(m & lanemask_lt());
      const unsigned long long c0 = cb + incl - (unsigned long long)nch;
      // both lists are sized for the input's rows (louvain_create); a
      // vertex that finds no room keeps reading its whole row
      if ((int64_t)blk < L.sample_cap && (int64_t)(c0 + nch) <= L.chunk_cap) {
        at = (int32_t)blk;
        L.sample_n[at] = 0u;
        for (int64_t c = 0; c < nch; ++c) L.chunks[c0 + c] = make_int2((int)v, (int)c);
      } else {
        for (int64_t c = 0; c < nch; ++c)
          if ((int64_t)(c0 + c) < L.chunk_cap) L.chunks[c0 + c] = make_int2(-1, 0);
      }
    }
    L.sample_at[v] = at;
  }
}

__global__ void __launch_bounds__(256) k_sample_chunks(GView g, LearnArgs L, const Counters *ctr) {
  const unsigned long long total = ctr->sample_chunks;
  const long long nch = (long long)total < L.chunk_cap ? (long long)total : L.chunk_cap;
  for (long long q = blockIdx.x; q < nch; q += gridDim.x) {
    const int2 rec = L.chunks[q];
    const int32_t i = rec.x;
    if (i < 0) continue;
    const int64_t b = g.begin[i], e = g.end[i];
    const unsigned long long thr = ((unsigned long long)kSampleTarget << 32) / (unsigned long long)(e - b);
    const uint32_t salt = fmix32((uint32_t)i ^ kSampleSalt);
    const int32_t at = L.sample_at[i];
    const int64_t k0 = b + (int64_t)rec.y * kSampleChunk;
    const int64_t k1 = k0 + kSampleChunk < e ? k0 + kSampleChunk : e;
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      const int32_t j = __ldg(g.col + k);
      if (j != i && (unsigned long long)fmix32((uint32_t)j ^ salt) < thr) {
        const uint32_t pos = atomicAdd(L.sample_n + at, 1u);
        if (pos < (uint32_t)kSample) L.sample[(int64_t)at * kSample + pos] = j;
      }
    }
  }
}

// ---------------------------------------------------------------- pass init
// K (row sums on the first pass; given otherwise), Sigma' = K', C' = id,
// all vertices unprocessed; the maximum degree and the size bound of the hub
// tables (sum of pow2(2 min(deg, n')) over degrees > 32768) for the host.
template <int WK>
__global__ void __launch_bounds__(256) k_pass_init(GView g, int first_pass, int64_t *K, int64_t *Sigma,
                                                   int32_t *Cp, uint8_t *flag, Counters *ctr, float4 *feat,
                                                   uint32_t *seen, uint32_t *moved_at, uint8_t *vbin,
                                                   int group_max, int half_max, int warp_max, int64_t track_min) {
  unsigned long long md = 0, big_slots = 0, big_items = 0;
  const int lane = threadIdx.x & 31;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = g.begin[i], e = g.end[i];
    const unsigned long long deg = (unsigned long long)(e - b);
    if (deg > md) md = deg;
    if (vbin)
      vbin[i] = (uint8_t)((deg > 0 ? (unsigned)move_bin((int64_t)deg, group_max, half_max, warp_max) : kVbinNone) |
                          (track_min > 0 && (int64_t)deg >= track_min ? kVbinTracked : 0u));
    if (deg > (unsigned long long)kWideMaxDeg) {  // hubs of the global tables
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
    flag[i] = kFlagUnproc;
    if (feat) {
      feat[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      seen[i] = 0;
      moved_at[i] = 0;
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

// Every vertex unprocessed (bit kFlagUnproc set, the tracked bit kept).
__global__ void k_flag_all(uint8_t *flag, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] |= kFlagUnproc;
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
  constexpr size_t kWideSmem =
      (size_t)kXlCap * (sizeof(uint32_t) + sizeof(int32_t)) + (size_t)kWideOcc * sizeof(uint16_t);
  if (!attr_done) {
    cudaFuncSetAttribute(k_move_block<WK, 512, kBlockCap, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kBlockSmem);
    cudaFuncSetAttribute(k_move_wide<WK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWideSmem);
    attr_done = true;
  }
  if (a.sel_list) {
    LV_TIMED(prof, K_SELECT, s, k_select_list<<<num_sms * 4, 256, 0, s>>>(a));
  } else {
    LV_TIMED(prof, K_SELECT, s,
             k_select<<<grid_for((a.g.n + kSelVPT - 1) / kSelVPT, 256, num_sms, 8), 256, 0, s>>>(a));
    if (a.learn.enabled) LV_TIMED(prof, K_MLP_SELECT, s, k_mlp_select<<<num_sms * 4, 256, 0, s>>>(a));
  }
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
  LV_TIMED(prof, K_MOVE_XL, s, k_move_wide<WK><<<num_sms, 1024, kWideSmem, s>>>(a));  // one block per SM, work queue
  if (hubs) big_move_rounds(big, WK, num_sms, s, prof);
  if (conc)
    for (int k = 0; k < kSideStreams; ++k) {
      cudaEventRecord(side->join[k], side->s[k]);
      cudaStreamWaitEvent(s, side->join[k], 0);
    }
  if (!a.async_apply && !a.refine) LV_TIMED(prof, K_APPLY, s, k_apply<<<num_sms * 4, 256, 0, s>>>(a));
}

template <int WK>
void pass_init_t(const GView &g, int first, int64_t *K, int64_t *Sigma, int32_t *Cp, uint8_t *flag, Counters *ctr,
                 int num_sms, cudaStream_t s, const LearnArgs *learn, uint8_t *vbin, const Sched *sched) {
  float4 *feat = (learn && learn->record) ? learn->feat : nullptr;
  const bool rec = learn && learn->record;
  LV_LAUNCH(k_pass_init<WK><<<grid_for(g.n, 256, num_sms, 16), 256, 0, s>>>(g, first, K, Sigma, Cp, flag, ctr, feat,
                                                                             rec ? learn->seen : nullptr,
                                                                             rec ? learn->moved_at : nullptr, vbin,
                                                                             sched ? sched->group_max : 0,
                                                                             sched ? sched->half_max : 0,
                                                                             sched ? sched->warp_max : 0,
                                                                             (learn && learn->record) ? learn->min_degree
                                                                                                      : 0));
  if (rec) {
    cudaMemsetAsync(&ctr->sample_blocks, 0, 2 * sizeof(unsigned long long), s);
    LV_LAUNCH(k_sample_plan<<<grid_for(g.n, 256, num_sms, 8), 256, 0, s>>>(g, *learn, ctr));
    LV_LAUNCH(k_sample_chunks<<<num_sms * 8, 256, 0, s>>>(g, *learn, ctr));
  }
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

void flag_all(uint8_t *flag, int64_t n, int num_sms, cudaStream_t s) {
  if (n <= 0) return;
  LV_LAUNCH(k_flag_all<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(flag, n));
}

void iota_i32(int32_t *x, int64_t n, int num_sms, cudaStream_t s) {
  if (n <= 0) return;
  LV_LAUNCH(k_iota<<<grid_for(n, 256, num_sms, 16), 256, 0, s>>>(x, n));
}

const char *const kKernelNames[K_NUM_KERNELS] = {
    "select", "move_thread", "move_warp", "move_mid", "move_block", "move_hub", "apply", "pass_init",
    "comm_count", "comm_scatter", "merge_thread", "merge_warp", "merge_mid", "merge_block", "merge_big",
    "dendrogram", "modularity", "renumber", "move_hub_eval", "merge_big_emit", "mlp_select", "move_group", "move_wide", "merge_xl", "merge_group", "move_half"};

}  // namespace lv
