// Per-vertex features of the learned vertex-activity predictor and the
// trace recorder.  A vertex's features at selection time:
//   x0 = log2(1 + degree) / 24
//   x1 = K_{i->d} / K_i at its last evaluation (intra-community fraction)
//   x2 = (s(c*) - s(d)) / (2m K_i) at its last evaluation, in [-1, 1]
//        (-1 when it had no candidate community): the best-dQ margin
//   x3 = 1 if it moved at its last evaluation
//   x4 = iteration / MAX_ITERATIONS, x5 = pass / MAX_PASSES
//   x6 = Sigma of its community / 2m
//   x7 = min(1, neighbour moves since its last evaluation / degree)
// Features are valid from the second evaluation of a vertex in a pass on.
#pragma once
#include "internal.h"
#include "mlp.cuh"

namespace lv {

__device__ __forceinline__ void vertex_features(const GView &g, const int32_t *Cp, const int64_t *Sigma,
                                                long long two_m, const LearnArgs &L, int32_t i, float4 fv,
                                                float (&x)[kFeatures]) {
  const int64_t deg = g.end[i] - g.begin[i];
  x[0] = log2f(1.f + (float)deg) * (1.f / 24.f);
  x[1] = fv.x;
  x[2] = fv.y;
  x[3] = fv.z;
  x[4] = L.t_norm;
  x[5] = L.p_norm;
  x[6] = (float)Sigma[Cp[i]] / (float)two_m;
  x[7] = fminf(1.f, (float)L.marks[i] / (float)(deg > 0 ? deg : 1));
}

// After the decision for vertex i (community d, K_i, K_{i->d}, best
// candidate, s(d), moved): optionally record a trace sample with the features
// it had when selected and whether it moved, then store its new features.
__device__ __forceinline__ void learn_record(const LearnArgs &L, Counters *ctr, const GView &g, const int32_t *Cp,
                                             const int64_t *Sigma, long long two_m, int32_t i, long long Ki,
                                             long long Kid, long long best_s, int32_t best_c, long long s_d,
                                             bool moved) {
  if (!L.record) return;
  if (L.min_degree > 0 && g.end[i] - g.begin[i] < L.min_degree) return;  // no features below the predictor's degree
  const float4 old = L.feat[i];
  if (L.trace_x && old.w > 0.f && (fmix32((uint32_t)i ^ L.trace_salt) & 0xFFFFu) < L.trace_keep) {
    const unsigned long long pos = atomicAdd(&ctr->trace_count, 1ull);
    if ((int64_t)pos < L.trace_cap) {
      float x[kFeatures];
      vertex_features(g, Cp, Sigma, two_m, L, i, old, x);
#pragma unroll
      for (int k = 0; k < kFeatures; ++k) L.trace_x[pos * kFeatures + k] = x[k];
      L.trace_y[pos] = moved ? 1.f : 0.f;
    }
  }
  float4 nv;
  nv.x = Ki > 0 ? (float)Kid / (float)Ki : 0.f;
  if (best_c == 0x7FFFFFFF || Ki == 0) {
    nv.y = -1.f;
  } else {
    const float m = (float)((double)(best_s - s_d) / ((double)two_m * (double)Ki));
    nv.y = fminf(1.f, fmaxf(-1.f, m));
  }
  nv.z = moved ? 1.f : 0.f;
  nv.w = 1.f;
  L.feat[i] = nv;
  L.marks[i] = 0;
}

// A mover's neighbour j: marked unprocessed (vertex pruning, bit kFlagUnproc
// of its flag byte) and, when features are kept, the move counts for j's
// next evaluation.  Moves go to marks_next, which the next selection folds
// into marks, so a decision never sees marks that change while its bucket
// runs.  When only vertices of some minimum degree keep features, their
// flag bytes carry kFlagTracked (set at pass start): the byte is read and
// written back, one sector as for the plain store, and only tracked
// neighbours pay the atomic.
__device__ __forceinline__ void mark_neighbour(uint8_t *flag, const LearnArgs &L, int32_t j) {
  if (L.record && L.min_degree > 0) {
    const uint8_t f = flag[j];
    flag[j] = (uint8_t)(f | kFlagUnproc);
    if (f & kFlagTracked) atomicAdd(L.marks_next + j, 1u);
  } else {
    flag[j] = kFlagUnproc;
    if (L.record) atomicAdd(L.marks_next + j, 1u);
  }
}

}  // namespace lv
