// Big items on sm_103a: hub vertices of the local-moving phase (Algorithm 5)
// and large communities of the aggregation phase (Algorithm 6) of arXiv
// 2501.19004: vertices of degree above 32768 (smaller ones fit a block's or
// a cluster's shared memory) and communities whose members hold more than
// 8192 entries.
//
// The paper gives such items a thread block each (Sec. 4.3.4).  On skewed
// graphs one item can hold hundreds of millions of entries, so here an item's
// entries are cut into chunks of 4096 that all blocks of the grid share:
//   k_big_plan    table offsets and chunk counts of every item (one block);
//   k_big_accum   each block pre-aggregates one chunk in shared memory
//                 (hot keys summed across the warp first), then adds the
//                 chunk's distinct keys into the item's global table and
//                 lists every slot it claims;
//   k_big_plan2   (aggregation) slices over the occupied-slot lists;
//   k_big_eval    (moving) blocks scan table slices: argmax of Eq. 2 per
//                 slice, clearing the slots as they go;
//   k_big_decide  (moving) one block per hub reduces its slices, decides and
//                 re-marks the neighbours;
//   k_big_emit    (aggregation) blocks take slices of occupied slots and
//                 append the super-edges to the community's row, clearing
//                 the slots.
// For aggregation an item's entries are the concatenated rows of its member
// vertices, located through the member-degree prefix (community-vertex CSR).
#include <climits>

#include "internal.h"
#include "learn.cuh"
#include "tables.cuh"

namespace lv {
namespace {

constexpr int kNT = 512;
constexpr unsigned kFull = 0xFFFFFFFFu;
enum { MODE_MOVE = 0, MODE_MERGE = 1 };

__device__ __forceinline__ uint32_t table_cap(int64_t tot, int64_t keyspace) {
  return (uint32_t)big_table_cap((uint64_t)tot, (uint64_t)keyspace);
}

// Items of round r: [rstart[r], rstart[r + 1]); table offset of item k inside
// the workspace: toff[k] - r * window.
struct RoundRange {
  int64_t k0, k1, base;
};
__device__ __forceinline__ RoundRange round_range(const BigArgs &a, int r) {
  RoundRange rr;
  rr.k0 = a.ws.rstart[r];
  rr.k1 = a.ws.rstart[r + 1];
  rr.base = (int64_t)r * a.window;
  return rr;
}

template <int MODE>
__global__ void __launch_bounds__(1024) k_big_plan(BigArgs a) {
  __shared__ long long sc0[33], sc1[33], sc2[33];
  const int64_t nb = (int64_t)*a.count;
  long long c_slots = 0, c_ch = 0, c_ev = 0;
  unsigned long long members = 0;
  for (int64_t base = 0; base < nb; base += 1024) {
    const int64_t k = base + threadIdx.x;
    long long tot = 0, cap = 0, nch = 0, nev = 0;
    if (k < nb) {
      const int32_t it = a.items[k];
      if (MODE == MODE_MOVE) {
        tot = a.g.end[it] - a.g.begin[it];
      } else {
        tot = a.oend[it] - a.obegin[it];  // row capacity = total member degree
        a.oend[it] = a.obegin[it];        // becomes the append cursor
        members += (unsigned long long)a.kcnt[it];
      }
      a.ws.tot[k] = tot;
      a.ws.ocnt[k] = 0;
      cap = table_cap(tot, a.keyspace);
      nch = (tot + kBigChunk - 1) / kBigChunk;
      nev = (cap + kBigEvalSlots - 1) / kBigEvalSlots;
    }
    long long t0, t1, t2;
    const long long e0 = block_scan_ex<1024>(cap, sc0, &t0);
    const long long e1 = block_scan_ex<1024>(nch, sc1, &t1);
    const long long e2 = block_scan_ex<1024>(nev, sc2, &t2);
    if (k < nb) {
      a.ws.toff[k] = c_slots + e0;
      a.ws.cpre[k] = c_ch + e1;
      if (MODE == MODE_MOVE) a.ws.epre[k] = c_ev + e2;
    }
    c_slots += t0;
    c_ch += t1;
    c_ev += t2;
  }
  if (MODE == MODE_MERGE) {
    members = warp_sum_u(members);
    if ((threadIdx.x & 31) == 0 && members) atomicAdd(&a.ctr->mg_work[kBigBin][1], members);
  }
  // rounds: item k belongs to round toff[k] / window; rstart holds the
  // pass's bound of rounds, the host launches the rounds these items need,
  // and the workspace holds the window plus the largest table
  const bool fits = c_slots <= (long long)a.rounds * a.window && (MODE == MODE_MERGE || c_ev <= a.ws.parts);
  __syncthreads();
  for (int64_t k = threadIdx.x; k <= nb; k += 1024) {
    const int64_t rk = k < nb ? a.ws.toff[k] / a.window : a.rounds;
    const int64_t rp = k > 0 ? a.ws.toff[k - 1] / a.window : -1;
    for (int64_t r = rp + 1; r <= rk && r <= a.rounds; ++r) a.ws.rstart[r] = fits ? k : nb;
  }
  if (threadIdx.x == 0) {
    if (!fits) {
      atomicOr(&a.ctr->error, (unsigned long long)ERR_HASH);
      for (int64_t r = 0; r <= a.rounds; ++r) a.ws.rstart[r] = nb;  // nothing runs
    }
    *a.ws.nrounds = fits ? (c_slots + a.window - 1) / a.window : 0;
    a.ws.toff[nb] = c_slots;
    a.ws.cpre[nb] = c_ch;
    a.ws.epre[nb] = MODE == MODE_MOVE ? c_ev : 0;
    if (MODE == MODE_MERGE) atomicAdd(&a.ctr->mg_work[kBigBin][0], (unsigned long long)nb);
  }
}

// Emission slices of round r (aggregation): kBigEvalSlots occupied slots
// each, a prefix over the round's items stored in epre[k0 .. k1].
__global__ void __launch_bounds__(1024) k_big_plan2(BigArgs a, int r) {
  __shared__ long long sc[33];
  const RoundRange rr = round_range(a, r);
  long long c_ev = 0;
  for (int64_t base = rr.k0; base < rr.k1; base += 1024) {
    const int64_t k = base + threadIdx.x;
    const long long nev = k < rr.k1 ? (long long)((a.ws.ocnt[k] + kBigEvalSlots - 1) / kBigEvalSlots) : 0;
    long long t;
    const long long e = block_scan_ex<1024>(nev, sc, &t);
    if (k < rr.k1) a.ws.epre[k] = c_ev + e;
    c_ev += t;
  }
  if (threadIdx.x == 0) a.ws.epre[rr.k1] = c_ev;  // total of the round
}

// Gather kRun entries of an item's entry sequence below xe: positions x,
// x + stride, ... for a hub's row (coalesced across threads), consecutive
// positions x, x + 1, ... for a community's member rows (one member search
// per run).
template <int MODE, int WK>
__device__ __forceinline__ void gather_item(const BigArgs &a, int32_t it, int64_t x, int64_t stride, int64_t xe,
                                            int32_t (&kk)[kRun], uint32_t (&ww)[kRun]) {
#pragma unroll
  for (int u = 0; u < kRun; ++u) {
    kk[u] = kEmpty;
    ww[u] = 0;
  }
  if (MODE == MODE_MOVE) {
    const int64_t b = a.g.begin[it];
    int32_t jj[kRun];
#pragma unroll
    for (int u = 0; u < kRun; ++u) {
      jj[u] = -2;
      const int64_t p = x + u * stride;
      if (p < xe) {
        jj[u] = __ldg(a.g.col + b + p);
        ww[u] = load_w<WK>(a.g.w, b + p);
      }
    }
#pragma unroll
    for (int u = 0; u < kRun; ++u) kk[u] = (jj[u] >= 0 && jj[u] != it) ? a.Cp[jj[u]] : kEmpty;
  } else {
    if (x >= xe) return;
    const int64_t m0 = a.kcoff[it];
    const int64_t base = a.obegin[it];  // = mprefix[m0]
    int64_t t = m0 + upper_index(a.mprefix + m0, a.kcnt[it], base + x);
    int64_t mstart = a.mprefix[t];
    int32_t v = a.members[t];
    int64_t rb = a.g.begin[v], rlen = a.g.end[v] - rb;
    int32_t jj[kRun];
    int64_t ee[kRun];
#pragma unroll
    for (int u = 0; u < kRun; ++u) {
      jj[u] = -2;
      if (x + u < xe) {
        int64_t pos = base + x + u;
        while (pos >= mstart + rlen) {  // next member with entries
          ++t;
          mstart = a.mprefix[t];
          v = a.members[t];
          rb = a.g.begin[v];
          rlen = a.g.end[v] - rb;
        }
        ee[u] = rb + (pos - mstart);
        jj[u] = __ldg(a.g.col + ee[u]);
        ww[u] = load_w<WK>(a.g.w, ee[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kRun; ++u) kk[u] = jj[u] >= 0 ? a.Cp[jj[u]] : kEmpty;
  }
}

template <int MODE, int WK>
__global__ void __launch_bounds__(kNT, 3) k_big_accum(BigArgs a, int r) {
  extern __shared__ uint32_t dyn[];
  int32_t *skeys = (int32_t *)dyn;
  uint32_t *svals = dyn + kBigSmemSlots;
  const RoundRange rr = round_range(a, r);
  const int64_t g0 = a.ws.cpre[rr.k0], g1 = a.ws.cpre[rr.k1];
  unsigned long long entries = 0;
  for (int s = threadIdx.x; s < kBigSmemSlots; s += kNT) {
    skeys[s] = kEmpty;
    svals[s] = 0;
  }
  __syncthreads();
  for (int64_t g = g0 + blockIdx.x; g < g1; g += gridDim.x) {
    const int64_t k = rr.k0 + upper_index(a.ws.cpre + rr.k0, rr.k1 - rr.k0, g);
    const int32_t it = a.items[k];
    const int64_t tot = a.ws.tot[k];
    const int64_t x0 = (g - a.ws.cpre[k]) * kBigChunk;
    const int64_t x1 = x0 + kBigChunk < tot ? x0 + kBigChunk : tot;
    int32_t kk[kRun];
    uint32_t ww[kRun];
    if (MODE == MODE_MOVE) {
      gather_item<MODE, WK>(a, it, x0 + threadIdx.x, kNT, x1, kk, ww);
    } else {
      const int64_t xs = x0 + (int64_t)threadIdx.x * kRun;
      gather_item<MODE, WK>(a, it, xs, 1, xs + kRun < x1 ? xs + kRun : x1, kk, ww);
    }
    if (threadIdx.x == 0) entries += (unsigned long long)(x1 - x0);
#pragma unroll
    for (int u = 0; u < kRun; ++u) {
      if (MODE == MODE_MERGE) {  // community rows repeat keys a lot: sum equal keys across the warp first
        warp_insert_sm(skeys, svals, kBigSmemSlots - 1, kk[u], ww[u], a.ctr);
      } else if (kk[u] != kEmpty) {
        sm_insert(skeys, svals, kBigSmemSlots - 1, kk[u], ww[u], a.ctr);
      }
    }
    __syncthreads();
    const int64_t toff = a.ws.toff[k] - rr.base;
    const uint32_t gcap = table_cap(tot, a.keyspace);
    unsigned long long *tab = a.ws.tab + toff;
    // the chunk's distinct keys go to the item's global table: every thread
    // first reads the home slots of several keys (independent loads in
    // flight), then claims or adds to each.
    // When aggregating, claimed slots are appended to the item's list with
    // one atomic per warp (emission then visits occupied slots only).
    constexpr int kPer = 4;  // keys in flight per thread
    for (int s0 = 0; s0 < kBigSmemSlots; s0 += kPer * kNT) {
      int32_t key[kPer];
      uint32_t wv[kPer], home[kPer];
      unsigned long long cur[kPer];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int s = s0 + u * kNT + threadIdx.x;
        key[u] = skeys[s];
        wv[u] = svals[s];
        skeys[s] = kEmpty;
        svals[s] = 0;
        cur[u] = 0ull;
        home[u] = 0;
        if (key[u] != kEmpty) {
          home[u] = slot_in_range(key[u], gcap);
          cur[u] = __ldcg(tab + home[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        int64_t slot = -1;
        if (key[u] != kEmpty) slot = gm_insert_packed_from(tab, gcap, home[u], cur[u], key[u], wv[u], a.ctr);
        if (MODE == MODE_MOVE) continue;
        const unsigned claimed = __ballot_sync(kFull, slot >= 0);
        if (claimed) {
          const int lane = threadIdx.x & 31, leader = __ffs(claimed) - 1;
          unsigned long long base = 0;
          if (lane == leader) base = atomicAdd(a.ws.ocnt + k, (unsigned long long)__popc(claimed));
          base = __shfl_sync(kFull, base, leader);
          if (slot >= 0) a.ws.occ[toff / 2 + (int64_t)(base + __popc(claimed & lanemask_lt()))] = (int32_t)slot;
        }
      }
    }
    __syncthreads();
  }
  unsigned long long w[1] = {entries};
  flush_work(w, MODE == MODE_MOVE ? &a.ctr->mv_work[kBigBin][1] : &a.ctr->mg_work[kBigBin][2]);
}

// Moving: per table slice, the best candidate (score, then lowest id) and the
// weight to the vertex's own community; slots are cleared.  Hub tables are
// at least a quarter full, so slices are scanned sequentially.
__global__ void __launch_bounds__(kNT) k_big_eval(BigArgs a, int r) {
  const RoundRange rr = round_range(a, r);
  const int64_t g0 = a.ws.epre[rr.k0], g1 = a.ws.epre[rr.k1];
  unsigned long long distinct = 0;
  for (int64_t g = g0 + blockIdx.x; g < g1; g += gridDim.x) {
    const int64_t k = rr.k0 + upper_index(a.ws.epre + rr.k0, rr.k1 - rr.k0, g);
    const int32_t i = a.items[k];
    const int64_t cap = table_cap(a.ws.tot[k], a.keyspace);
    const int64_t s0 = (g - a.ws.epre[k]) * kBigEvalSlots;
    const int64_t s1 = s0 + kBigEvalSlots < cap ? s0 + kBigEvalSlots : cap;
    unsigned long long *tab = a.ws.tab + (a.ws.toff[k] - rr.base);
    const int32_t d = a.Cp[i];
    const long long Ki = a.K[i];
    const long long tm = vertex_two_m(a.batch, a.two_m, i);
    long long best_s = LLONG_MIN, Kid = 0;
    int32_t best_c = INT_MAX;
    // 8 slots per thread per round: all loads issued before use
    constexpr int kPer = 8;
    for (int64_t r0 = s0; r0 < s1; r0 += kPer * kNT) {
      unsigned long long pv[kPer];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int64_t s = r0 + u * kNT + threadIdx.x;
        pv[u] = s < s1 ? __ldcg(tab + s) : 0ull;
      }
      long long sig[kPer];
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        const int32_t c = packed_key(pv[u]);
        sig[u] = (pv[u] != 0ull && c != d) ? a.Sigma[c] : 0;
      }
#pragma unroll
      for (int u = 0; u < kPer; ++u) {
        if (pv[u] == 0ull) continue;
        tab[r0 + u * kNT + threadIdx.x] = 0ull;
        const int32_t c = packed_key(pv[u]);
        const long long v = packed_val(pv[u]);
        if (c == d) {
          Kid = v;
          continue;
        }
        ++distinct;
        const long long sc = tm * v - Ki * sig[u];
        if (better(sc, c, best_s, best_c)) {
          best_s = sc;
          best_c = c;
        }
      }
    }
    block_argmax_sum<kNT>(best_s, best_c, Kid);
    if (threadIdx.x == 0) {
      a.ws.part_s[g] = best_s;
      a.ws.part_c[g] = best_c;
      a.ws.part_kid[g] = (unsigned long long)Kid;
    }
  }
  unsigned long long w[1] = {distinct};
  flush_work(w, &a.ctr->mv_work[kBigBin][2]);
}

// Moving: one block per hub reduces its slices and applies Algorithm 5's
// decision; movers re-mark their neighbours.
__global__ void __launch_bounds__(kNT) k_big_decide(BigArgs a, int r) {
  __shared__ int32_t s_target;
  const RoundRange rr = round_range(a, r);
  unsigned long long glo = 0, ghi = 0, gm = 0;
  unsigned long long work[3] = {0, 0, 0};  // vertices, movers, mover entries
  for (int64_t k = rr.k0 + blockIdx.x; k < rr.k1; k += gridDim.x) {
    const int32_t i = a.items[k];
    long long best_s = LLONG_MIN, Kid = 0;
    int32_t best_c = INT_MAX;
    for (int64_t p = a.ws.epre[k] + threadIdx.x; p < a.ws.epre[k + 1]; p += kNT) {
      const long long s = a.ws.part_s[p];
      const int32_t c = a.ws.part_c[p];
      Kid += (long long)a.ws.part_kid[p];
      if (better(s, c, best_s, best_c)) {
        best_s = s;
        best_c = c;
      }
    }
    block_argmax_sum<kNT>(best_s, best_c, Kid);
    const int64_t b = a.g.begin[i], e = a.g.end[i];
    if (threadIdx.x == 0) {
      const int32_t d = a.Cp[i];
      long long s_d = 0;
      const long long tm = vertex_two_m(a.batch, a.two_m, i);
      const int32_t t = finish_decision(tm, a.Sigma, a.iter ? (int)a.iter[1] : a.pickless, d, a.K[i], Kid, best_s, best_c, glo, ghi, gm, &s_d);
      learn_record(a.learn, a.ctr, a.g, a.Cp, a.Sigma, a.two_m, i, a.K[i], Kid, best_s, best_c, s_d, t >= 0);
      if (t >= 0) batch_gain(a.batch, i, best_s, s_d);
      work[0] += 1;
      if (t >= 0) {
        work[1] += 1;
        work[2] += (unsigned long long)(e - b);
        const unsigned long long pos = atomicAdd(&a.ctr->movers, 1ull);
        emit_move(a.async_apply, a.apply_Cp, a.K, a.apply_Sigma, a.mv_vertex, a.mv_target, pos, i, t);
      }
      s_target = t;
    }
    __syncthreads();
    if (s_target >= 0)
      mark_neighbours(a.flag, a.g.col, b, e, threadIdx.x, kNT, i);
    __syncthreads();
  }
  flush_gains(glo, ghi, gm, a.ctr);
  unsigned long long w0[1] = {work[0]};
  flush_work(w0, &a.ctr->mv_work[kBigBin][0]);
  unsigned long long w1[2] = {work[1], work[2]};
  flush_work(w1, &a.ctr->mv_work[kBigBin][3]);
}

// Aggregation: append every occupied slot of a slice to the community's row
// (super-edge (c, key, weight)); slots are cleared.
__global__ void __launch_bounds__(kNT) k_big_emit(BigArgs a, int r) {
  __shared__ unsigned long long s_base;
  const RoundRange rr = round_range(a, r);
  const int64_t total = a.ws.epre[rr.k1];  // round-local prefix (k_big_plan2)
  unsigned long long written = 0;
  for (int64_t g = blockIdx.x; g < total; g += gridDim.x) {
    const int64_t k = rr.k0 + upper_index(a.ws.epre + rr.k0, rr.k1 - rr.k0, g);
    const int32_t c = a.items[k];
    const int64_t nocc = (int64_t)a.ws.ocnt[k];
    const int64_t p0 = (g - a.ws.epre[k]) * kBigEvalSlots;
    const int64_t p1 = p0 + kBigEvalSlots < nocc ? p0 + kBigEvalSlots : nocc;
    const int64_t toff = a.ws.toff[k] - rr.base;
    unsigned long long *tab = a.ws.tab + toff;
    const int32_t *occ = a.ws.occ + toff / 2;
    if (threadIdx.x == 0) {
      s_base = atomicAdd((unsigned long long *)(a.oend + c), (unsigned long long)(p1 - p0));
      written += (unsigned long long)(p1 - p0);
    }
    __syncthreads();
    for (int64_t p = p0 + threadIdx.x; p < p1; p += kNT) {
      const int32_t s = occ[p];
      const unsigned long long pos = s_base + (unsigned long long)(p - p0);
      const unsigned long long pv = __ldcg(tab + s);
      a.ocol[pos] = packed_key(pv);
      a.ow[pos] = packed_val(pv);
      tab[s] = 0ull;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && written) {
    atomicAdd(&a.ctr->nnz_out, written);
    atomicAdd(&a.ctr->mg_work[kBigBin][3], written);
  }
}

template <int MODE>
void big_plan(const BigArgs &b, cudaStream_t s, KernelProf *prof) {
  const int k_rest = MODE == MODE_MOVE ? K_MOVE_HUB_EVAL : K_MERGE_BIG_EMIT;
  if (prof) prof->begin(k_rest, s);
  LV_LAUNCH(k_big_plan<MODE><<<1, 1024, 0, s>>>(b));
  if (prof) prof->end(k_rest, s);
  if (b.static_rounds) return;
  cudaMemcpyAsync(b.h_rounds, b.ws.nrounds, sizeof(long long), cudaMemcpyDeviceToHost, s);
  cudaEventRecord(b.plan_done, s);
}

template <int MODE, int WK>
void big_rounds(const BigArgs &b, int num_sms, cudaStream_t s, KernelProf *prof) {
  const int k_acc = MODE == MODE_MOVE ? K_MOVE_HUB : K_MERGE_BIG;
  const int k_rest = MODE == MODE_MOVE ? K_MOVE_HUB_EVAL : K_MERGE_BIG_EMIT;
  static bool attr_done = false;
  constexpr size_t kSmem = (size_t)kBigSmemSlots * (sizeof(int32_t) + sizeof(uint32_t));
  if (!attr_done) {
    cudaFuncSetAttribute(k_big_accum<MODE, WK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    attr_done = true;
  }
  long long nr = b.rounds;  // rounds beyond the items' need find no items
  if (!b.static_rounds) {
    cudaEventSynchronize(b.plan_done);
    nr = *b.h_rounds < b.rounds ? *b.h_rounds : b.rounds;
  }
  for (int r = 0; r < nr; ++r) {
    LV_TIMED(prof, k_acc, s, k_big_accum<MODE, WK><<<num_sms * b.accum_blocks, kNT, kSmem, s>>>(b, r));
    if (prof) prof->begin(k_rest, s);
    if (MODE == MODE_MERGE) LV_LAUNCH(k_big_plan2<<<1, 1024, 0, s>>>(b, r));
    if (MODE == MODE_MOVE) {
      LV_LAUNCH(k_big_eval<<<num_sms * 3, kNT, 0, s>>>(b, r));
      LV_LAUNCH(k_big_decide<<<num_sms * 2, kNT, 0, s>>>(b, r));
    } else {
      LV_LAUNCH(k_big_emit<<<num_sms * 3, kNT, 0, s>>>(b, r));
    }
    if (prof) prof->end(k_rest, s);
  }
}

}  // namespace

void big_move_plan(const BigArgs &b, cudaStream_t s, KernelProf *prof) { big_plan<MODE_MOVE>(b, s, prof); }

void big_move_rounds(const BigArgs &b, int wkind, int num_sms, cudaStream_t s, KernelProf *prof) {
  if (wkind == W_UNIT) big_rounds<MODE_MOVE, W_UNIT>(b, num_sms, s, prof);
  else big_rounds<MODE_MOVE, W_U32>(b, num_sms, s, prof);
}

void big_merge(const BigArgs &b, int wkind, int num_sms, cudaStream_t s, KernelProf *prof) {
  big_plan<MODE_MERGE>(b, s, prof);
  if (wkind == W_UNIT) big_rounds<MODE_MERGE, W_UNIT>(b, num_sms, s, prof);
  else big_rounds<MODE_MERGE, W_U32>(b, num_sms, s, prof);
}

}  // namespace lv
