// Per-vertex features of the learned vertex-activity predictor and the
// trace recorder.  A vertex's features at selection time:
//   x0 = log2(1 + degree) / 24
//   x1 = K_{i->d} / K_i at its last evaluation (intra-community fraction)
//   x2 = (s(c*) - s(d)) / (2m K_i) at its last evaluation, in [-1, 1]
//        (-1 when it had no candidate community): the best-dQ margin
//   x3 = 1 if it moved at its last evaluation
//   x4 = iteration / MAX_ITERATIONS, x5 = pass / MAX_PASSES
//   x6 = Sigma of its community / 2m
//   x7 = fraction of its sampled neighbours that moved since its last
//        evaluation: a neighbour counts when the bucket of its last move is
//        not earlier than the bucket of the vertex's last evaluation.  The
//        sample is the whole row up to kSample entries; for longer rows, the
//        neighbours j with fmix32(j ^ fmix32(i ^ kSampleSalt)) below
//        2^32 kSampleTarget / degree, a set that does not depend on the order
//        of the row (the whole row again if more than kSample qualify).
// Features are valid from the second evaluation of a vertex in a pass on.
#pragma once
#include "internal.h"
#include "mlp.cuh"

namespace lv {

constexpr uint32_t kSampleSalt = 0x5BD1E995u;

// Feature x7 of vertex i (see above).
__device__ __forceinline__ float neighbour_move_fraction(const GView &g, const LearnArgs &L, int32_t i) {
  const uint32_t since = L.seen[i];
  unsigned moved = 0, total = 0;
  const int32_t at = L.sample_at[i];
  const uint32_t ns = at >= 0 ? L.sample_n[at] : 0u;
  if (at < 0 || ns > (uint32_t)kSample) {
    for (int64_t k = g.begin[i], e = g.end[i]; k < e; ++k) {
      const int32_t j = __ldg(g.col + k);
      if (j == i) continue;
      const uint32_t m = L.moved_at[j];
      ++total;
      moved += (m != 0u && m >= since) ? 1u : 0u;
    }
  } else {
    const int32_t *sp = L.sample + (int64_t)at * kSample;
    for (uint32_t p = 0; p < ns; ++p) {
      const uint32_t m = L.moved_at[sp[p]];
      moved += (m != 0u && m >= since) ? 1u : 0u;
    }
    total = ns;
  }
  return total ? (float)moved / (float)total : 0.f;
}

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
  x[7] = neighbour_move_fraction(g, L, i);
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
  L.seen[i] = L.stamp;
}

// The neighbours col[k] (k = b + t, b + t + stride, ... < e) of mover i are
// marked unprocessed (vertex pruning, Sec. 4.1.6): one plain byte store each.
__device__ __forceinline__ void mark_neighbours(uint8_t *flag, const int32_t *col, int64_t b, int64_t e, int64_t t,
                                                int64_t stride, int32_t i) {
  for (int64_t k = b + t; k < e; k += stride) {
    const int32_t j = __ldg(col + k);
    if (j != i) flag[j] = kFlagUnproc;
  }
}

}  // namespace lv
