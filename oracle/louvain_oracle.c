/*
 * Louvain oracle: a plain, slow CPU restatement of the method of
 * "CPU vs. GPU for Community Detection: Performance Insights from
 * GVE-Louvain and nu-Louvain" (arXiv 2501.19004).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes, in the paper's order and notation:
 *   - the pass loop of Algorithm 1 / Algorithm 4 (Sec. 4.2.1, Appendix);
 *   - the local-moving phase of Algorithm 2 / Algorithm 5 (Sec. 4.2.2),
 *     with vertex pruning (Sec. 4.1.6) and Pick-Less mode (Sec. 4.3.1);
 *   - the aggregation phase of Algorithm 3 / Algorithm 6 (Sec. 4.2.3);
 *   - modularity, Eq. 1, and delta-modularity, Eq. 2 (Sec. 3.2);
 *   - optionally the refinement phase of the Leiden algorithm (Traag,
 *     Waltman and van Eck 2019), which Sec. 5.2 and Sec. 6 expect the
 *     paper's findings to carry over to; the greedy, bucketed form used
 *     here is described at leiden_refine below.
 *
 * The paper's algorithms move vertices asynchronously.  This oracle instead
 * fixes one deterministic semi-synchronous schedule: in every iteration the
 * vertices are split into B buckets by a hash of (vertex, pass, iteration);
 * bucket by bucket, every unprocessed vertex of the bucket is marked
 * processed, all of them decide against the same snapshot of C' and Sigma',
 * and then all moves are applied.  Eq. 2 is compared exactly in integers:
 * 2m^2 * dQ_{i:d->c} = s(c) - s(d) with s(c) = 2m K_{i->c} - K_i Sigma_c and
 * s(d) = 2m K_{i->d} - K_i (Sigma_d - K_i); the argmax takes the lowest
 * community id among equal scores and a move needs s(c*) > s(d).
 * All sums are exact (__int128); nothing here is a floating-point
 * approximation except the final conversions to double for the tolerance
 * tests and for Q, which take one rounding each.
 *
 * Everything is plain: the neighbour-community map of a vertex is built by
 * sorting its (community, weight) pairs and summing runs.  The only
 * concurrency is an OpenMP loop over vertices of a bucket (each decision
 * reads the snapshot only) and over communities in aggregation (each writes
 * its own output row); results do not depend on the thread count.
 */
#include <limits.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

/* ---- configuration and outputs (mirrors the library's run parameters) ---- */
typedef struct {
  int32_t max_passes;            /* MAX_PASSES, Sec. 4.3 item (2): 10 */
  int32_t max_iterations;        /* MAX_ITERATIONS, Sec. 4.1.2: 20 */
  double tolerance;              /* initial tau, Sec. 4.1.4: 0.01 */
  double tolerance_drop;         /* TOLERANCE_DROP, Sec. 4.1.3: 10 */
  double aggregation_tolerance;  /* tau_agg, Sec. 4.1.5: 0.8 */
  int32_t pickless_period;       /* rho of Pick-Less mode, Sec. 4.3.1: 4 (0 = off) */
  int32_t buckets;               /* B of the deterministic schedule: 4 */
  uint64_t schedule_seed;        /* seed of the bucket hash */
  int32_t check_invariants;      /* verify sum(Sigma') == 2m after every bucket */
  int32_t num_threads;           /* 0 = OpenMP default */
  int32_t refine;                /* 1: Leiden refinement before aggregation (see or_refine) */
} or_config;

enum { OR_OK = 0, OR_E_INVAL = 1, OR_E_NOMEM = 2, OR_E_INVARIANT = 3 };

/* per iteration record: [evaluated, moves, gain_hi, gain_lo] (gain = sum of
 * s(c*) - s(d) over the moves, exact, split as hi*2^64 + lo) */
#define OR_ITER_FIELDS 4
/* per pass record: [n', nnz', l_i, |Gamma|, Q_num_hi, Q_num_lo] where Q_num is
 * 2m*S_in - S_tot of (G', C') after the moving phase */
#define OR_PASS_FIELDS 6

/* ---- current graph G': compact CSR with 64-bit weights ---- */
typedef struct {
  int64_t n, nnz;
  int64_t *off;
  int32_t *col;
  int64_t *w;
} graph_t;

typedef struct { int32_t c; int64_t w; } pair_t;

static int cmp_pair(const void *a, const void *b) {
  int32_t x = ((const pair_t *)a)->c, y = ((const pair_t *)b)->c;
  return (x > y) - (x < y);
}

static void graph_free(graph_t *g) {
  free(g->off);
  free(g->col);
  free(g->w);
  memset(g, 0, sizeof(*g));
}

static int graph_from_input(graph_t *g, int64_t n, const int64_t *off, const int32_t *col,
                            const int32_t *w) {
  int64_t nnz = off[n];
  g->n = n;
  g->nnz = nnz;
  g->off = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  g->col = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
  g->w = (int64_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int64_t));
  if (!g->off || !g->col || !g->w) { graph_free(g); return OR_E_NOMEM; }
  memcpy(g->off, off, ((size_t)n + 1) * sizeof(int64_t));
  if (nnz) memcpy(g->col, col, (size_t)nnz * sizeof(int32_t));
  for (int64_t k = 0; k < nnz; ++k) g->w[k] = w ? (int64_t)w[k] : 1;
  return OR_OK;
}

/* ---- the bucket hash of the deterministic schedule ----
 * fmix32 is the MurmurHash3 finaliser (Appleby, MurmurHash3, public domain).
 * salt(p, t) = fmix32(fold(seed) ^ (((p << 8) | t) * 0x9E3779B1))
 * bucket(i)  = fmix32(i ^ salt(p, t)) mod B                                */
static uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

static uint32_t bucket_of(int64_t i, int32_t pass, int32_t iter, uint64_t seed, int32_t B) {
  uint32_t fold = (uint32_t)seed ^ (uint32_t)(seed >> 32);
  uint32_t pt = ((uint32_t)pass << 8) | ((uint32_t)iter & 0xFFu);
  uint32_t salt = fmix32(fold ^ (pt * 0x9E3779B1u));
  return fmix32((uint32_t)i ^ salt) % (uint32_t)B;
}

uint32_t or_fmix32(uint32_t h) { return fmix32(h); }
uint32_t or_bucket(int64_t i, int32_t pass, int32_t iter, uint64_t seed, int32_t B) {
  return bucket_of(i, pass, iter, seed, B);
}

/* ---- Eq. 2 in integers ----
 * 2m^2 * dQ_{i:d->c} = [2m K_{i->c} - K_i Sigma_c] - [2m K_{i->d} - K_i (Sigma_d - K_i)] */
static i128 score_other(int64_t two_m, int64_t K_ic, int64_t K_i, int64_t Sigma_c) {
  return (i128)two_m * K_ic - (i128)K_i * Sigma_c;
}
static i128 score_own(int64_t two_m, int64_t K_id, int64_t K_i, int64_t Sigma_d) {
  return (i128)two_m * K_id - (i128)K_i * (Sigma_d - K_i);
}

/* scanCommunities (Algorithm 2): the map c -> K_{i->c} over the edges of i,
 * skipping the self-loop unless self != 0.  Returned as sorted runs in buf;
 * the number of distinct communities is returned. */
static int64_t scan_communities(const graph_t *g, const int32_t *Cp, int64_t i, int self,
                                pair_t *buf) {
  int64_t k = 0;
  for (int64_t e = g->off[i]; e < g->off[i + 1]; ++e) {
    int64_t j = g->col[e];
    if (!self && j == i) continue;
    buf[k].c = Cp[j];
    buf[k].w = g->w[e];
    ++k;
  }
  if (k > 1) qsort(buf, (size_t)k, sizeof(pair_t), cmp_pair);
  int64_t r = 0;
  for (int64_t t = 0; t < k; ++t) {
    if (r > 0 && buf[r - 1].c == buf[t].c) buf[r - 1].w += buf[t].w;
    else buf[r++] = buf[t];
  }
  return r;
}

typedef struct { int32_t target; int32_t moves; i128 gain; } decision_t;

/* One vertex of the local-moving phase (Algorithm 5 body): choose the best
 * community linked to i against the snapshot (C', Sigma'), then apply the
 * "same community" and Pick-Less rejections. */
static decision_t decide(const graph_t *g, const int32_t *Cp, const int64_t *K, const int64_t *Sigma,
                         int64_t two_m, int64_t i, int pickless, pair_t *buf) {
  decision_t out = {Cp[i], 0, 0};
  int64_t r = scan_communities(g, Cp, i, 0, buf);
  int32_t d = Cp[i];
  int64_t K_i = K[i], K_id = 0;
  for (int64_t t = 0; t < r; ++t)
    if (buf[t].c == d) K_id = buf[t].w;
  i128 s_d = score_own(two_m, K_id, K_i, Sigma[d]);
  int have = 0;
  int32_t best_c = -1;
  i128 best_s = 0;
  for (int64_t t = 0; t < r; ++t) {
    int32_t c = buf[t].c;
    if (c == d) continue;
    i128 s = score_other(two_m, buf[t].w, K_i, Sigma[c]);
    if (!have || s > best_s || (s == best_s && c < best_c)) {
      have = 1;
      best_s = s;
      best_c = c;
    }
  }
  if (!have || !(best_s > s_d)) return out;   /* c* = C'[i]: stay */
  if (pickless && best_c > d) return out;     /* Pick-Less rejects c* > C'[i] */
  out.target = best_c;
  out.moves = 1;
  out.gain = best_s - s_d;
  return out;
}

static int64_t max_degree(const graph_t *g) {
  int64_t m = 0;
  for (int64_t i = 0; i < g->n; ++i) {
    int64_t d = g->off[i + 1] - g->off[i];
    if (d > m) m = d;
  }
  return m;
}

static int nthreads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
static int thread_id(void) {
#ifdef _OPENMP
  return omp_get_thread_num();
#else
  return 0;
#endif
}

/* The local-moving phase (Algorithm 2 / 5) under the bucket schedule.
 * Returns l_i, the number of iterations performed. */
static int louvain_move(const graph_t *g, int32_t *Cp, const int64_t *K, int64_t *Sigma,
                        uint8_t *unprocessed, int64_t two_m, double tau, int32_t pass,
                        const or_config *cfg, int64_t *iter_stats, int *status) {
  const int64_t n = g->n;
  const int T = nthreads();
  const int64_t md = max_degree(g);
  pair_t **bufs = (pair_t **)calloc((size_t)T, sizeof(pair_t *));
  int64_t *A = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  decision_t *dec = (decision_t *)malloc((size_t)(n ? n : 1) * sizeof(decision_t));
  int ok = bufs && A && dec;
  for (int t = 0; ok && t < T; ++t) {
    bufs[t] = (pair_t *)malloc((size_t)(md ? md : 1) * sizeof(pair_t));
    ok = bufs[t] != NULL;
  }
  int li_done = cfg->max_iterations;
  if (!ok) { *status = OR_E_NOMEM; goto out; }
  const i128 den2 = (i128)two_m * two_m;  /* (2m)^2 = 2 * (2m^2) */
  for (int li = 0; li < cfg->max_iterations; ++li) {
    const int rho = cfg->pickless_period;
    const int pickless = rho > 0 && ((li + rho / 2) % rho) == 0;
    i128 dQ = 0;  /* total 2m^2 * delta-modularity of this iteration */
    int64_t evaluated = 0, moves = 0;
    for (int32_t b = 0; b < cfg->buckets; ++b) {
      /* snapshot: unprocessed vertices of this bucket, marked processed */
      int64_t na = 0;
      for (int64_t i = 0; i < n; ++i)
        if (unprocessed[i] && (int32_t)bucket_of(i, pass, li, cfg->schedule_seed, cfg->buckets) == b) {
          unprocessed[i] = 0;
          A[na++] = i;
        }
      evaluated += na;
      /* decide against the snapshot */
#pragma omp parallel for schedule(dynamic, 64)
      for (int64_t a = 0; a < na; ++a)
        dec[a] = decide(g, Cp, K, Sigma, two_m, A[a], pickless, bufs[thread_id()]);
      /* apply: Sigma' updates, C' updates, remark neighbours */
      for (int64_t a = 0; a < na; ++a) {
        if (!dec[a].moves) continue;
        int64_t i = A[a];
        int32_t d = Cp[i], c = dec[a].target;
        Sigma[d] -= K[i];
        Sigma[c] += K[i];
        Cp[i] = c;
        dQ += dec[a].gain;
        ++moves;
        for (int64_t e = g->off[i]; e < g->off[i + 1]; ++e)
          if (g->col[e] != i) unprocessed[g->col[e]] = 1;
      }
      if (cfg->check_invariants) {
        i128 tot = 0;
        for (int64_t c = 0; c < n; ++c) tot += Sigma[c];
        if (tot != two_m) { *status = OR_E_INVARIANT; goto out; }
      }
    }
    if (iter_stats) {
      int64_t *r = iter_stats + ((int64_t)pass * cfg->max_iterations + li) * OR_ITER_FIELDS;
      r[0] = evaluated;
      r[1] = moves;
      r[2] = (int64_t)(dQ >> 64);
      r[3] = (int64_t)(uint64_t)dQ;
    }
    /* delta-modularity total: dQ / (2m^2) = (2 dQ) / (2m)^2 */
    double total = den2 ? (double)(2 * dQ) / (double)den2 : 0.0;
    if (total <= tau) { li_done = li + 1; break; }
  }
out:
  if (bufs) for (int t = 0; t < T; ++t) free(bufs[t]);
  free(bufs);
  free(A);
  free(dec);
  return li_done;
}

#define OR_REFINE_BUCKETS_PER_B 4

/* ---- Leiden refinement (Traag, Waltman & van Eck 2019, the refinement of
 * the partition P that local moving produced; the paper's Sec. 5.2 and
 * Sec. 6 expect its findings to extend to Leiden) ----
 *
 * Greedy and deterministic, in the same bucket form as local moving:
 *   - The refined partition starts as singletons: Cr[v] = v, Sr[v] = K_v.
 *   - A vertex v may move only while it is a singleton, and only if it is
 *     well connected to its community C = P(v):
 *       2m K_{v->C} >= K_v (Sigma_C - K_v)
 *     where K_{v->C} sums v's edges to the other members of C.
 *   - One sweep over R buckets of (v, pass, iteration 255); a whole run
 *     uses R = 4B (OR_REFINE_BUCKETS_PER_B), so that fewer decisions are
 *     simultaneous than in local moving: Leiden visits vertices one at a
 *     time, each seeing the merges made before it.  In a bucket,
 *     every such vertex decides against the snapshot (Cr, Sr) exactly as in
 *     local moving, but sees only neighbours inside its own community C: it
 *     picks the refined community T (within C) with the largest
 *     s(T) = 2m K_{v->T} - K_v Sr[T], lowest id on ties, and moves iff
 *     s(T) > 0 (its own singleton scores 0).  No Pick-Less.
 *   - A vertex that any decision of the bucket chose as its target stays
 *     where it is and can no longer move; the other movers are applied.
 *     So no mover is ever the target of another, and every refined
 *     community keeps the id of one of its members (the target the others
 *     joined, which never moves).
 * Every merge needs K_{v->T} > 0, so refined communities are connected
 * subsets of the communities of P.  Leiden's randomised choice among the
 * merges that do not lower the quality is replaced by the best one. */

/* G' restricted to the edges inside the communities of `bound`, self-loops
 * dropped (rows keep their order). */
static int filter_to_bounds(const graph_t *g, const int32_t *bound, graph_t *out) {
  out->n = g->n;
  out->off = (int64_t *)malloc((size_t)(g->n + 1) * sizeof(int64_t));
  if (!out->off) return OR_E_NOMEM;
  int64_t k = 0;
  out->off[0] = 0;
  for (int64_t i = 0; i < g->n; ++i) {
    for (int64_t e = g->off[i]; e < g->off[i + 1]; ++e)
      if (g->col[e] != i && bound[g->col[e]] == bound[i]) ++k;
    out->off[i + 1] = k;
  }
  out->nnz = k;
  out->col = (int32_t *)malloc((size_t)(k ? k : 1) * sizeof(int32_t));
  out->w = (int64_t *)malloc((size_t)(k ? k : 1) * sizeof(int64_t));
  if (!out->col || !out->w) return OR_E_NOMEM;
  k = 0;
  for (int64_t i = 0; i < g->n; ++i)
    for (int64_t e = g->off[i]; e < g->off[i + 1]; ++e)
      if (g->col[e] != i && bound[g->col[e]] == bound[i]) {
        out->col[k] = g->col[e];
        out->w[k] = g->w[e];
        ++k;
      }
  return OR_OK;
}

/* Refined partition Cr (raw ids: a member's vertex id) of G' under P =
 * bound, whose community totals are Sigma_b; K are the vertex weights; the
 * sweep runs over `rbuckets` buckets of the schedule's hash. */
static int leiden_refine(const graph_t *g, const int32_t *bound, const int64_t *K, const int64_t *Sigma_b,
                         int64_t two_m, int32_t pass, int32_t rbuckets, uint64_t seed, int32_t *Cr) {
  const int64_t n = g->n;
  graph_t F = {0, 0, NULL, NULL, NULL};
  int st = filter_to_bounds(g, bound, &F);
  const int T = nthreads();
  int64_t *Sr = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  uint8_t *elig = (uint8_t *)malloc((size_t)(n ? n : 1));
  uint8_t *chosen = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
  int64_t *A = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  decision_t *dec = (decision_t *)malloc((size_t)(n ? n : 1) * sizeof(decision_t));
  pair_t **bufs = (pair_t **)calloc((size_t)T, sizeof(pair_t *));
  const int64_t md = max_degree(g);
  if (st || !Sr || !elig || !chosen || !A || !dec || !bufs) st = OR_E_NOMEM;
  for (int t = 0; !st && t < T; ++t) {
    bufs[t] = (pair_t *)malloc((size_t)(md ? md : 1) * sizeof(pair_t));
    if (!bufs[t]) st = OR_E_NOMEM;
  }
  if (st) goto out;
  for (int64_t v = 0; v < n; ++v) {
    int64_t kin = 0;
    for (int64_t e = F.off[v]; e < F.off[v + 1]; ++e) kin += F.w[e];
    elig[v] = (i128)two_m * kin >= (i128)K[v] * (Sigma_b[bound[v]] - K[v]);
    Cr[v] = (int32_t)v;
    Sr[v] = K[v];
  }
  for (int32_t b = 0; b < rbuckets; ++b) {
    int64_t na = 0;
    for (int64_t v = 0; v < n; ++v)
      if (elig[v] && !chosen[v] && (int32_t)bucket_of(v, pass, 255, seed, rbuckets) == b)
        A[na++] = v;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t a = 0; a < na; ++a)
      dec[a] = decide(&F, Cr, K, Sr, two_m, A[a], 0, bufs[thread_id()]);
    for (int64_t a = 0; a < na; ++a)
      if (dec[a].moves) chosen[dec[a].target] = 1;
    for (int64_t a = 0; a < na; ++a) {
      const int64_t v = A[a];
      if (!dec[a].moves || chosen[v]) continue;
      const int32_t t = dec[a].target;
      Sr[v] -= K[v];
      Sr[t] += K[v];
      Cr[v] = t;
    }
  }
out:
  if (bufs) for (int t = 0; t < T; ++t) free(bufs[t]);
  free(bufs);
  free(Sr);
  free(elig);
  free(chosen);
  free(A);
  free(dec);
  graph_free(&F);
  return st;
}

/* Renumber communities densely, keeping their order (the new id of c is the
 * number of used ids below c).  Returns |Gamma|. */
static int64_t renumber(int32_t *x, int64_t len, int64_t id_space) {
  int32_t *newid = (int32_t *)malloc((size_t)(id_space ? id_space : 1) * sizeof(int32_t));
  if (!newid) return -1;
  for (int64_t c = 0; c < id_space; ++c) newid[c] = 0;
  for (int64_t i = 0; i < len; ++i) newid[x[i]] = 1;
  int64_t run = 0;
  for (int64_t c = 0; c < id_space; ++c) {
    int32_t used = newid[c];
    newid[c] = (int32_t)run;
    run += used;
  }
  for (int64_t i = 0; i < len; ++i) x[i] = newid[x[i]];
  free(newid);
  return run;
}

static int64_t count_distinct(const int32_t *x, int64_t len, int64_t id_space) {
  uint8_t *seen = (uint8_t *)calloc((size_t)(id_space ? id_space : 1), 1);
  if (!seen) return -1;
  int64_t r = 0;
  for (int64_t i = 0; i < len; ++i)
    if (!seen[x[i]]) { seen[x[i]] = 1; ++r; }
  free(seen);
  return r;
}

/* The aggregation phase (Algorithm 3 / 6): community vertices by count, scan
 * and scatter (in vertex order), then one super-vertex per community whose
 * edges are the summed weights to every linked community, self-loops kept
 * (scanCommunities with self = true).  Rows of G'' are sorted by id.
 * Cp must be dense in [0, ncomm). */
static int louvain_aggregate(const graph_t *g, const int32_t *Cp, int64_t ncomm, graph_t *out) {
  const int64_t n = g->n;
  int64_t *coff = (int64_t *)calloc((size_t)ncomm + 1, sizeof(int64_t));
  int64_t *cv = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  int64_t *ctot = (int64_t *)calloc((size_t)ncomm + 1, sizeof(int64_t));
  int64_t *rowlen = (int64_t *)calloc((size_t)ncomm + 1, sizeof(int64_t));
  memset(out, 0, sizeof(*out));
  if (!coff || !cv || !ctot || !rowlen) goto nomem;
  /* countCommunityVertices + exclusiveScan + scatter */
  for (int64_t i = 0; i < n; ++i) coff[Cp[i] + 1]++;
  for (int64_t c = 0; c < ncomm; ++c) coff[c + 1] += coff[c];
  {
    int64_t *cur = (int64_t *)malloc((size_t)(ncomm ? ncomm : 1) * sizeof(int64_t));
    if (!cur) goto nomem;
    memcpy(cur, coff, (size_t)ncomm * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) cv[cur[Cp[i]]++] = i;
    free(cur);
  }
  /* communityTotalDegree: an upper bound on each super-vertex's degree */
  for (int64_t c = 0; c < ncomm; ++c)
    for (int64_t k = coff[c]; k < coff[c + 1]; ++k) ctot[c] += g->off[cv[k] + 1] - g->off[cv[k]];
  /* first sweep: distinct linked communities per community */
  {
    int ok = 1;
#pragma omp parallel
    {
      pair_t *buf = NULL;
      int64_t cap = 0;
#pragma omp for schedule(dynamic, 16)
      for (int64_t c = 0; c < ncomm; ++c) {
        if (!ok) continue;
        if (ctot[c] > cap) {
          free(buf);
          cap = ctot[c];
          buf = (pair_t *)malloc((size_t)cap * sizeof(pair_t));
          if (!buf) { ok = 0; cap = 0; continue; }
        }
        int64_t k = 0;
        for (int64_t t = coff[c]; t < coff[c + 1]; ++t) {
          int64_t i = cv[t];
          for (int64_t e = g->off[i]; e < g->off[i + 1]; ++e) {
            buf[k].c = Cp[g->col[e]];
            buf[k].w = g->w[e];
            ++k;
          }
        }
        if (k > 1) qsort(buf, (size_t)k, sizeof(pair_t), cmp_pair);
        int64_t r = 0;
        for (int64_t t = 0; t < k; ++t) {
          if (r > 0 && buf[r - 1].c == buf[t].c) buf[r - 1].w += buf[t].w;
          else buf[r++] = buf[t];
        }
        rowlen[c] = r;
      }
      free(buf);
    }
    if (!ok) goto nomem;
  }
  out->n = ncomm;
  out->off = (int64_t *)malloc(((size_t)ncomm + 1) * sizeof(int64_t));
  if (!out->off) goto nomem;
  out->off[0] = 0;
  for (int64_t c = 0; c < ncomm; ++c) out->off[c + 1] = out->off[c] + rowlen[c];
  out->nnz = out->off[ncomm];
  out->col = (int32_t *)malloc((size_t)(out->nnz ? out->nnz : 1) * sizeof(int32_t));
  out->w = (int64_t *)malloc((size_t)(out->nnz ? out->nnz : 1) * sizeof(int64_t));
  if (!out->col || !out->w) goto nomem;
  /* second sweep: write the rows */
  {
    int ok = 1;
#pragma omp parallel
    {
      pair_t *buf = NULL;
      int64_t cap = 0;
#pragma omp for schedule(dynamic, 16)
      for (int64_t c = 0; c < ncomm; ++c) {
        if (!ok) continue;
        if (ctot[c] > cap) {
          free(buf);
          cap = ctot[c];
          buf = (pair_t *)malloc((size_t)cap * sizeof(pair_t));
          if (!buf) { ok = 0; cap = 0; continue; }
        }
        int64_t k = 0;
        for (int64_t t = coff[c]; t < coff[c + 1]; ++t) {
          int64_t i = cv[t];
          for (int64_t e = g->off[i]; e < g->off[i + 1]; ++e) {
            buf[k].c = Cp[g->col[e]];
            buf[k].w = g->w[e];
            ++k;
          }
        }
        if (k > 1) qsort(buf, (size_t)k, sizeof(pair_t), cmp_pair);
        int64_t r = 0;
        for (int64_t t = 0; t < k; ++t) {
          if (r > 0 && buf[r - 1].c == buf[t].c) buf[r - 1].w += buf[t].w;
          else buf[r++] = buf[t];
        }
        for (int64_t t = 0; t < r; ++t) {
          out->col[out->off[c] + t] = buf[t].c;
          out->w[out->off[c] + t] = buf[t].w;
        }
      }
      free(buf);
    }
    if (!ok) goto nomem;
  }
  free(coff);
  free(cv);
  free(ctot);
  free(rowlen);
  return OR_OK;
nomem:
  free(coff);
  free(cv);
  free(ctot);
  free(rowlen);
  graph_free(out);
  return OR_E_NOMEM;
}

/* Eq. 1 in integers: Q = (2m S_in - S_tot) / (2m)^2 with S_in the summed
 * weight of entries inside communities (sum of sigma_c) and S_tot the sum of
 * Sigma_c^2.  Membership ids must lie in [0, id_space). */
static int modularity_exact(const graph_t *g, const int32_t *C, int64_t id_space, i128 *num, i128 *den) {
  int64_t *Sig = (int64_t *)calloc((size_t)(id_space ? id_space : 1), sizeof(int64_t));
  if (!Sig) return OR_E_NOMEM;
  i128 s_in = 0, two_m = 0;
  for (int64_t i = 0; i < g->n; ++i)
    for (int64_t e = g->off[i]; e < g->off[i + 1]; ++e) {
      two_m += g->w[e];
      Sig[C[i]] += g->w[e];
      if (C[g->col[e]] == C[i]) s_in += g->w[e];
    }
  i128 s_tot = 0;
  for (int64_t c = 0; c < id_space; ++c) s_tot += (i128)Sig[c] * Sig[c];
  free(Sig);
  *num = two_m * s_in - s_tot;
  *den = two_m * two_m;
  return OR_OK;
}

static void put128(int64_t *dst, i128 v) {
  dst[0] = (int64_t)(v >> 64);
  dst[1] = (int64_t)(uint64_t)v;
}

static int validate_input(int64_t n, const int64_t *off, const int32_t *col, const int32_t *w) {
  if (n < 0 || !off) return OR_E_INVAL;
  if (off[0] != 0) return OR_E_INVAL;
  for (int64_t i = 0; i < n; ++i)
    if (off[i + 1] < off[i]) return OR_E_INVAL;
  for (int64_t k = 0; k < off[n]; ++k) {
    if (col[k] < 0 || col[k] >= n) return OR_E_INVAL;
    if (w && w[k] <= 0) return OR_E_INVAL;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------
 * Exported entry points
 * ---------------------------------------------------------------------- */

/* Modularity (Eq. 1) of `membership` (ids in [0, n)) on the input graph.
 * num_out/den_out receive the exact numerator and denominator as (hi, lo). */
int or_modularity(int64_t n, const int64_t *off, const int32_t *col, const int32_t *w,
                  const int32_t *membership, int64_t *num_out, int64_t *den_out, double *q) {
  if (validate_input(n, off, col, w)) return OR_E_INVAL;
  for (int64_t i = 0; i < n; ++i)
    if (membership[i] < 0 || membership[i] >= (n ? n : 1)) return OR_E_INVAL;
  graph_t g;
  if (graph_from_input(&g, n, off, col, w)) return OR_E_NOMEM;
  i128 num, den;
  int st = modularity_exact(&g, membership, n, &num, &den);
  graph_free(&g);
  if (st) return st;
  if (num_out) put128(num_out, num);
  if (den_out) put128(den_out, den);
  *q = den ? (double)num / (double)den : 0.0;
  return OR_OK;
}

/* 2m^2 * (change of Q) predicted by Eq. 2 for moving vertex i from its
 * community d = membership[i] to community c (c == d gives 0).  Sigma and K
 * are derived from the membership.  result = s(c) - s(d) as (hi, lo). */
int or_delta_modularity(int64_t n, const int64_t *off, const int32_t *col, const int32_t *w,
                        const int32_t *membership, int64_t i, int32_t c, int64_t *result) {
  if (validate_input(n, off, col, w) || i < 0 || i >= n || c < 0 || c >= n) return OR_E_INVAL;
  graph_t g;
  if (graph_from_input(&g, n, off, col, w)) return OR_E_NOMEM;
  int64_t *K = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  int64_t *Sig = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  pair_t *buf = (pair_t *)malloc((size_t)(g.nnz ? g.nnz : 1) * sizeof(pair_t));
  if (!K || !Sig || !buf) { free(K); free(Sig); free(buf); graph_free(&g); return OR_E_NOMEM; }
  int64_t two_m = 0;
  for (int64_t v = 0; v < n; ++v) {
    for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e) K[v] += g.w[e];
    Sig[membership[v]] += K[v];
    two_m += K[v];
  }
  int64_t r = scan_communities(&g, membership, i, 0, buf);
  int32_t d = membership[i];
  int64_t K_id = 0, K_ic = 0;
  for (int64_t t = 0; t < r; ++t) {
    if (buf[t].c == d) K_id = buf[t].w;
    if (buf[t].c == c) K_ic = buf[t].w;
  }
  i128 s_d = score_own(two_m, K_id, K[i], Sig[d]);
  i128 s_c = (c == d) ? s_d : score_other(two_m, K_ic, K[i], Sig[c]);
  put128(result, s_c - s_d);
  free(K);
  free(Sig);
  free(buf);
  graph_free(&g);
  return OR_OK;
}

/* One decision of the local-moving phase for vertex i against the snapshot
 * (membership, Sigma derived from it).  out = [moves, target, gain_hi, gain_lo]. */
int or_decide(int64_t n, const int64_t *off, const int32_t *col, const int32_t *w,
              const int32_t *membership, int64_t i, int32_t pickless, int64_t *out) {
  if (validate_input(n, off, col, w) || i < 0 || i >= n) return OR_E_INVAL;
  graph_t g;
  if (graph_from_input(&g, n, off, col, w)) return OR_E_NOMEM;
  int64_t *K = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  int64_t *Sig = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  pair_t *buf = (pair_t *)malloc((size_t)(g.nnz ? g.nnz : 1) * sizeof(pair_t));
  if (!K || !Sig || !buf) { free(K); free(Sig); free(buf); graph_free(&g); return OR_E_NOMEM; }
  int64_t two_m = 0;
  for (int64_t v = 0; v < n; ++v) {
    for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e) K[v] += g.w[e];
    Sig[membership[v]] += K[v];
    two_m += K[v];
  }
  decision_t dd = decide(&g, membership, K, Sig, two_m, i, pickless, buf);
  out[0] = dd.moves;
  out[1] = dd.target;
  put128(out + 2, dd.gain);
  free(K);
  free(Sig);
  free(buf);
  graph_free(&g);
  return OR_OK;
}

/* Aggregation of the input graph by a dense membership in [0, ncomm).
 * Two calls: with col_out == NULL only *nnz_out is set; then the caller
 * provides off_out[ncomm+1], col_out[nnz], w_out[nnz]. */
int or_aggregate(int64_t n, const int64_t *off, const int32_t *col, const int32_t *w,
                 const int32_t *membership, int64_t ncomm, int64_t *nnz_out, int64_t *off_out,
                 int32_t *col_out, int64_t *w_out) {
  if (validate_input(n, off, col, w) || ncomm < 0) return OR_E_INVAL;
  for (int64_t i = 0; i < n; ++i)
    if (membership[i] < 0 || membership[i] >= ncomm) return OR_E_INVAL;
  graph_t g, s;
  if (graph_from_input(&g, n, off, col, w)) return OR_E_NOMEM;
  int st = louvain_aggregate(&g, membership, ncomm, &s);
  graph_free(&g);
  if (st) return st;
  *nnz_out = s.nnz;
  if (col_out) {
    memcpy(off_out, s.off, ((size_t)ncomm + 1) * sizeof(int64_t));
    if (s.nnz) {
      memcpy(col_out, s.col, (size_t)s.nnz * sizeof(int32_t));
      memcpy(w_out, s.w, (size_t)s.nnz * sizeof(int64_t));
    }
  }
  graph_free(&s);
  return OR_OK;
}

/* The Leiden refinement alone (leiden_refine): the refined partition of
 * the input graph under the partition `bound` (ids in [0, n)), with vertex
 * weights from the rows, at pass index `pass` of the bucket hash, in one
 * sweep over `buckets` buckets (a whole run's sweep uses 4B).
 * refined_out [n]: raw refined ids (a member's vertex id). */
int or_refine(int64_t n, const int64_t *off, const int32_t *col, const int32_t *w, const int32_t *bound,
              int32_t pass, uint64_t seed, int32_t buckets, int32_t *refined_out) {
  if (validate_input(n, off, col, w) || buckets < 1) return OR_E_INVAL;
  for (int64_t i = 0; i < n; ++i)
    if (bound[i] < 0 || bound[i] >= n) return OR_E_INVAL;
  graph_t G;
  if (graph_from_input(&G, n, off, col, w)) return OR_E_NOMEM;
  int64_t *K = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
  int64_t *Sb = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
  int st = (K && Sb) ? OR_OK : OR_E_NOMEM;
  int64_t two_m = 0;
  for (int64_t i = 0; !st && i < n; ++i) {
    for (int64_t e = G.off[i]; e < G.off[i + 1]; ++e) K[i] += G.w[e];
    Sb[bound[i]] += K[i];
    two_m += K[i];
  }
  if (!st) st = leiden_refine(&G, bound, K, Sb, two_m, pass, buckets, seed, refined_out);
  free(K);
  free(Sb);
  graph_free(&G);
  return st;
}

/* The whole method (Algorithm 1 / 4); with cfg->refine, the Leiden form:
 * after local moving, the partition C' (P) is refined (leiden_refine), the
 * refined partition is aggregated, and the next pass starts every
 * super-vertex in its community of P (represented by the smallest
 * super-vertex of that community).  The low-shrink test then compares the
 * number of refined communities with n'; the final memberships are P's.
 *   membership_out [n]: final community of every input vertex, renumbered
 *                       densely in order of first id.
 *   iter_stats [max_passes * max_iterations * OR_ITER_FIELDS] or NULL
 *   pass_stats [max_passes * OR_PASS_FIELDS] or NULL
 *   summary [8]: passes performed, |Gamma| final, Q_num(hi, lo), Q_den(hi, lo),
 *                2m, status of the last pass-loop exit (0 max passes,
 *                1 converged l_i <= 1, 2 low shrink)
 *   q_out: final modularity as double. */
int or_louvain(int64_t n, const int64_t *off, const int32_t *col, const int32_t *w,
               const or_config *cfg, int32_t *membership_out, int64_t *iter_stats,
               int64_t *pass_stats, int64_t *summary, double *q_out) {
  if (!cfg || cfg->max_passes < 0 || cfg->max_iterations < 1 || cfg->max_iterations > 255 ||
      cfg->buckets < 1 || cfg->buckets > 65536 || cfg->pickless_period < 0 || cfg->refine < 0 || cfg->refine > 1)
    return OR_E_INVAL;
  if (validate_input(n, off, col, w)) return OR_E_INVAL;
#ifdef _OPENMP
  if (cfg->num_threads > 0) omp_set_num_threads(cfg->num_threads);
#endif
  if (iter_stats)
    memset(iter_stats, 0, (size_t)cfg->max_passes * cfg->max_iterations * OR_ITER_FIELDS * sizeof(int64_t));
  if (pass_stats) memset(pass_stats, 0, (size_t)cfg->max_passes * OR_PASS_FIELDS * sizeof(int64_t));
  int st = OR_OK;
  graph_t G;  /* G' */
  if (graph_from_input(&G, n, off, col, w)) return OR_E_NOMEM;
  int64_t two_m = 0;
  for (int64_t k = 0; k < G.nnz; ++k) two_m += G.w[k];
  int32_t *C = membership_out;
  for (int64_t i = 0; i < n; ++i) C[i] = (int32_t)i;
  int32_t *Cp = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
  int64_t *K = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  int64_t *Sigma = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  uint8_t *unproc = (uint8_t *)malloc((size_t)(n ? n : 1));
  /* Leiden: refined partition, next pass's initial partition, and the
   * smallest super-vertex of every community of P */
  int32_t *Cr = NULL, *init = NULL, *rep = NULL;
  if (cfg->refine) {
    Cr = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    init = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    rep = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    if (!Cr || !init || !rep) { st = OR_E_NOMEM; goto done; }
  }
  if (!Cp || !K || !Sigma || !unproc) { st = OR_E_NOMEM; goto done; }
  double tau = cfg->tolerance;
  int pending = 0;  /* C' of the last pass not yet looked up into C */
  int passes = 0, exit_reason = 0;
  for (int32_t lp = 0; lp < cfg->max_passes; ++lp) {
    const int64_t np = G.n;
    /* Sigma' <- K' <- vertexWeights(G'); C' <- [0 .. |V'|) */
    for (int64_t i = 0; i < np; ++i) {
      int64_t s = 0;
      for (int64_t e = G.off[i]; e < G.off[i + 1]; ++e) s += G.w[e];
      K[i] = s;
      Sigma[i] = s;
      Cp[i] = (int32_t)i;
      unproc[i] = 1;  /* mark all vertices as unprocessed */
    }
    if (cfg->refine && lp > 0) {  /* Leiden: start from the previous pass's P */
      for (int64_t i = 0; i < np; ++i) Sigma[i] = 0;
      for (int64_t i = 0; i < np; ++i) {
        Cp[i] = init[i];
        Sigma[init[i]] += K[i];
      }
    }
    int li = louvain_move(&G, Cp, K, Sigma, unproc, two_m, tau, lp, cfg, iter_stats, &st);
    if (st) goto done;
    ++passes;
    int64_t gamma = count_distinct(Cp, np, np);
    if (gamma < 0) { st = OR_E_NOMEM; goto done; }
    if (pass_stats) {
      int64_t *r = pass_stats + (int64_t)lp * OR_PASS_FIELDS;
      i128 qn, qd;
      if (modularity_exact(&G, Cp, np, &qn, &qd)) { st = OR_E_NOMEM; goto done; }
      r[0] = np;
      r[1] = G.nnz;
      r[2] = li;
      r[3] = gamma;
      put128(r + 4, qn);
    }
    if (li <= 1) { pending = 1; exit_reason = 1; break; }             /* globally converged */
    /* the partition to aggregate: C' (Louvain) or its refinement (Leiden) */
    int32_t *agg = Cp;
    int64_t nagg = gamma;
    if (cfg->refine) {
      st = leiden_refine(&G, Cp, K, Sigma, two_m, lp, OR_REFINE_BUCKETS_PER_B * cfg->buckets,
                         cfg->schedule_seed, Cr);
      if (st) goto done;
      agg = Cr;
      nagg = count_distinct(Cr, np, np);
      if (nagg < 0) { st = OR_E_NOMEM; goto done; }
    }
    if ((double)nagg / (double)np > cfg->aggregation_tolerance) {     /* low shrink */
      pending = 1;
      exit_reason = 2;
      break;
    }
    if (renumber(agg, np, np) < 0) { st = OR_E_NOMEM; goto done; }
    for (int64_t v = 0; v < n; ++v) C[v] = agg[C[v]];                 /* dendrogram lookup */
    if (cfg->refine) {  /* next pass starts every super-vertex in its community of P */
      for (int64_t c = 0; c < np; ++c) rep[c] = INT32_MAX;
      for (int64_t v = 0; v < np; ++v)
        if (Cr[v] < rep[Cp[v]]) rep[Cp[v]] = Cr[v];
      for (int64_t v = 0; v < np; ++v) init[Cr[v]] = rep[Cp[v]];
    }
    graph_t H;
    st = louvain_aggregate(&G, agg, nagg, &H);
    if (st) goto done;
    graph_free(&G);
    G = H;
    tau /= cfg->tolerance_drop;                                       /* threshold scaling */
  }
  if (pending)
    for (int64_t v = 0; v < n; ++v) C[v] = Cp[C[v]];
  if (!pending && cfg->refine && passes > 0)  /* pass cap: the last pass's P, not its refinement */
    for (int64_t v = 0; v < n; ++v) C[v] = init[C[v]];
  {
    int64_t gamma = renumber(C, n, n);
    if (gamma < 0) { st = OR_E_NOMEM; goto done; }
    graph_t G0;
    if (graph_from_input(&G0, n, off, col, w)) { st = OR_E_NOMEM; goto done; }
    i128 qn, qd;
    st = modularity_exact(&G0, C, n, &qn, &qd);
    graph_free(&G0);
    if (st) goto done;
    if (summary) {
      summary[0] = passes;
      summary[1] = gamma;
      put128(summary + 2, qn);
      put128(summary + 4, qd);
      summary[6] = two_m;
      summary[7] = exit_reason;
    }
    if (q_out) *q_out = qd ? (double)qn / (double)qd : 0.0;
  }
done:
  free(Cr);
  free(init);
  free(rep);
  free(Cp);
  free(K);
  free(Sigma);
  free(unproc);
  graph_free(&G);
  return st;
}

int or_num_threads(void) { return nthreads(); }
