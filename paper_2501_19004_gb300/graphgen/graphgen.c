/*
 * Seeded synthetic graph generators (planted-partition SBM, R-MAT, 2D grid
 * with long-range edges).  These produce the *inputs* of the Louvain method;
 * nothing in this file computes any part of the method itself.
 *
 * Every random number is a pure function of (seed, counter): SplitMix64
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014; the finaliser constants are Vigna's published ones), so the
 * output is identical for any thread count.  Undirected edges are stored in
 * both directions; self-loops are dropped; duplicate edges are merged; each
 * CSR row is sorted by column.  Weights of weighted graphs are a hash of the
 * unordered vertex pair, so duplicates agree and merging is order-free.
 *
 * Built as a small shared library and called through ctypes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int64_t n;
  int64_t nnz;
  int64_t *off;   /* [n+1] */
  int32_t *col;   /* [nnz] */
  int32_t *w;     /* [nnz] or NULL (unit weights) */
} gg_graph;

static inline uint64_t sm64(uint64_t seed, uint64_t idx) {
  uint64_t z = seed + (idx + 1u) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t gg_splitmix64(uint64_t seed, uint64_t idx) { return sm64(seed, idx); }

/* uniform double in [0, 1) with 53 random bits */
static inline double unif53(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

typedef struct { uint64_t seed; int lo, hi; } weight_rule;

static inline int32_t pair_weight(const weight_rule *wr, int64_t n, int64_t a, int64_t b) {
  int64_t lo = a < b ? a : b, hi = a < b ? b : a;
  uint64_t h = sm64(wr->seed, (uint64_t)lo * (uint64_t)n + (uint64_t)hi);
  return (int32_t)(wr->lo + (int64_t)(h % (uint64_t)(wr->hi - wr->lo + 1)));
}

/* Build a symmetric, deduplicated, row-sorted CSR from an undirected pair
 * list (pu[k], pv[k]); pairs with pu==pv are skipped.  Frees pu/pv. */
static gg_graph *build_csr(int64_t n, int64_t np, uint32_t *pu, uint32_t *pv,
                           const weight_rule *wr) {
  gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
  if (!g) return NULL;
  g->n = n;
  int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!deg) { free(g); return NULL; }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < np; ++k) {
    if (pu[k] == pv[k]) continue;
    __atomic_fetch_add(&deg[pu[k]], 1, __ATOMIC_RELAXED);
    __atomic_fetch_add(&deg[pv[k]], 1, __ATOMIC_RELAXED);
  }
  int64_t *off = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!off) { free(deg); free(g); return NULL; }
  int64_t run = 0;
  for (int64_t i = 0; i < n; ++i) { off[i] = run; run += deg[i]; }
  off[n] = run;
  int32_t *col = (int32_t *)malloc((size_t)(run > 0 ? run : 1) * sizeof(int32_t));
  if (!col) { free(off); free(deg); free(g); return NULL; }
  for (int64_t i = 0; i < n; ++i) deg[i] = off[i]; /* reuse as cursor */
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < np; ++k) {
    uint32_t u = pu[k], v = pv[k];
    if (u == v) continue;
    int64_t a = __atomic_fetch_add(&deg[u], 1, __ATOMIC_RELAXED);
    int64_t b = __atomic_fetch_add(&deg[v], 1, __ATOMIC_RELAXED);
    col[a] = (int32_t)v;
    col[b] = (int32_t)u;
  }
  free(pu);
  free(pv);
  /* sort and dedup every row; deg[i] becomes the deduplicated degree */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) {
    int64_t s = off[i], e = off[i + 1];
    int64_t d = e - s;
    if (d > 1) qsort(col + s, (size_t)d, sizeof(int32_t), cmp_i32);
    int64_t k = 0;
    for (int64_t t = 0; t < d; ++t)
      if (k == 0 || col[s + t] != col[s + k - 1]) col[s + (k++)] = col[s + t];
    deg[i] = k;
  }
  /* compact in place (destinations never pass their sources) */
  int64_t pos = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t s = off[i], d = deg[i];
    if (pos != s && d > 0) memmove(col + pos, col + s, (size_t)d * sizeof(int32_t));
    off[i] = pos;
    pos += d;
  }
  off[n] = pos;
  free(deg);
  int32_t *shrunk = (int32_t *)realloc(col, (size_t)(pos > 0 ? pos : 1) * sizeof(int32_t));
  if (shrunk) col = shrunk;
  g->off = off;
  g->col = col;
  g->nnz = pos;
  g->w = NULL;
  if (wr) {
    g->w = (int32_t *)malloc((size_t)(pos > 0 ? pos : 1) * sizeof(int32_t));
    if (!g->w) { free(col); free(off); free(g); return NULL; }
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i)
      for (int64_t k = off[i]; k < off[i + 1]; ++k) g->w[k] = pair_weight(wr, n, i, col[k]);
  }
  return g;
}

void gg_free(gg_graph *g) {
  if (!g) return;
  free(g->off);
  free(g->col);
  free(g->w);
  free(g);
}

void gg_size(const gg_graph *g, int64_t *n, int64_t *nnz, int32_t *weighted) {
  *n = g->n;
  *nnz = g->nnz;
  *weighted = g->w != NULL;
}

void gg_copy(const gg_graph *g, int64_t *off, int32_t *col, int32_t *w) {
  memcpy(off, g->off, ((size_t)g->n + 1) * sizeof(int64_t));
  if (g->nnz) memcpy(col, g->col, (size_t)g->nnz * sizeof(int32_t));
  if (w && g->w && g->nnz) memcpy(w, g->w, (size_t)g->nnz * sizeof(int32_t));
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004): 2^scale vertices, edge_factor *
 * 2^scale samples; each sample picks one quadrant per level with
 * probabilities (a, b, c, 1-a-b-c), decided by comparing a 32-bit uniform
 * draw with integer thresholds.  No vertex relabelling. */
gg_graph *gg_rmat(int scale, int64_t edge_factor, double a, double b, double c,
                  uint64_t seed, int wlo, int whi) {
  if (scale < 1 || scale > 31 || edge_factor < 1) return NULL;
  int64_t n = (int64_t)1 << scale;
  int64_t ns = edge_factor * n;
  uint32_t *pu = (uint32_t *)malloc((size_t)ns * sizeof(uint32_t));
  uint32_t *pv = (uint32_t *)malloc((size_t)ns * sizeof(uint32_t));
  if (!pu || !pv) { free(pu); free(pv); return NULL; }
  const uint64_t TA = (uint64_t)(a * 4294967296.0);
  const uint64_t TB = TA + (uint64_t)(b * 4294967296.0);
  const uint64_t TC = TB + (uint64_t)(c * 4294967296.0);
  const int draws = (scale + 1) / 2;
  const uint64_t s = sm64(seed, 0x524D4154ULL); /* "RMAT" sub-stream */
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < ns; ++k) {
    uint32_t u = 0, v = 0;
    for (int j = 0; j < draws; ++j) {
      uint64_t x = sm64(s, (uint64_t)k * (uint64_t)draws + (uint64_t)j);
      for (int h = 0; h < 2; ++h) {
        if (2 * j + h >= scale) break;
        uint64_t r = h ? (x >> 32) : (x & 0xFFFFFFFFULL);
        uint32_t ub = (r >= TB), vb = (r >= TA && r < TB) || (r >= TC);
        u = (u << 1) | ub;
        v = (v << 1) | vb;
      }
    }
    pu[k] = u;
    pv[k] = v;
  }
  weight_rule wr = {sm64(seed, 0x57474854ULL), wlo, whi};
  return build_csr(n, ns, pu, pv, (wlo == 1 && whi == 1) ? NULL : &wr);
}

/* Planted-partition SBM on n vertices in consecutive blocks of `block`
 * vertices (the last block takes the remainder).  Intra-block pairs are drawn
 * one by one with probability p_in.  Inter-block pairs are drawn with
 * probability p_out: one by one when direct != 0, otherwise by geometric
 * skipping over the n*n index space (Batagelj & Brandes, Phys. Rev. E 71,
 * 2005), keeping only u < v in different blocks. */
gg_graph *gg_sbm(int64_t n, int64_t block, double p_in, double p_out, uint64_t seed, int direct) {
  if (n < 1 || block < 1) return NULL;
  const uint64_t s_in = sm64(seed, 0x53424D31ULL), s_out = sm64(seed, 0x53424D32ULL);
  int64_t nblocks = (n + block - 1) / block;
  /* intra: count first so the pair list is sized exactly */
  int64_t cap = 1024;
  int64_t np = 0;
  uint32_t *pu = (uint32_t *)malloc((size_t)cap * sizeof(uint32_t));
  uint32_t *pv = (uint32_t *)malloc((size_t)cap * sizeof(uint32_t));
  if (!pu || !pv) { free(pu); free(pv); return NULL; }
#define PUSH(U, V)                                                                  \
  do {                                                                              \
    if (np == cap) {                                                                \
      cap *= 2;                                                                     \
      uint32_t *nu = (uint32_t *)realloc(pu, (size_t)cap * sizeof(uint32_t));       \
      uint32_t *nv = (uint32_t *)realloc(pv, (size_t)cap * sizeof(uint32_t));       \
      if (!nu || !nv) { free(nu ? nu : pu); free(nv ? nv : pv); return NULL; }      \
      pu = nu; pv = nv;                                                             \
    }                                                                               \
    pu[np] = (uint32_t)(U); pv[np] = (uint32_t)(V); ++np;                           \
  } while (0)
  for (int64_t bl = 0; bl < nblocks; ++bl) {
    int64_t lo = bl * block, hi = lo + block < n ? lo + block : n;
    for (int64_t u = lo; u < hi; ++u)
      for (int64_t v = u + 1; v < hi; ++v)
        if (unif53(sm64(s_in, (uint64_t)u * (uint64_t)n + (uint64_t)v)) < p_in) PUSH(u, v);
  }
  if (p_out > 0.0) {
    if (direct) {
      for (int64_t u = 0; u < n; ++u)
        for (int64_t v = u + 1; v < n; ++v)
          if (u / block != v / block &&
              unif53(sm64(s_out, (uint64_t)u * (uint64_t)n + (uint64_t)v)) < p_out)
            PUSH(u, v);
    } else {
      const double lq = log1p(-p_out);
      const uint64_t total = (uint64_t)n * (uint64_t)n;
      uint64_t idx = 0, draw = 0;
      for (;;) {
        double r = unif53(sm64(s_out, draw++));
        double skip = floor(log1p(-r) / lq);
        if (skip >= (double)(total - idx)) break;
        idx += (uint64_t)skip;
        int64_t u = (int64_t)(idx / (uint64_t)n), v = (int64_t)(idx % (uint64_t)n);
        if (u < v && u / block != v / block) PUSH(u, v);
        ++idx;
        if (idx >= total) break;
      }
    }
  }
#undef PUSH
  return build_csr(n, np, pu, pv, NULL);
}

/* Union of G planted-partition graphs (gg_sbm with the geometric-skip
 * sampler), generated in parallel one graph per thread: graph k owns the
 * vertices [vo[k], vo[k+1]) and its columns are shifted by vo[k].  vo_out
 * receives G + 1 offsets.  Identical to concatenating gg_sbm's outputs. */
gg_graph *gg_sbm_union(int64_t G, const int64_t *n, const int64_t *block, const double *p_in, const double *p_out,
                       const uint64_t *seed, int64_t *vo_out) {
  if (G < 1) return NULL;
  gg_graph **parts = (gg_graph **)calloc((size_t)G, sizeof(gg_graph *));
  int64_t *eo = (int64_t *)calloc((size_t)G + 1, sizeof(int64_t));
  if (!parts || !eo) { free(parts); free(eo); return NULL; }
  int fail = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t k = 0; k < G; ++k) {
    parts[k] = gg_sbm(n[k], block[k], p_in[k], p_out[k], seed[k], 0);
    if (!parts[k]) __atomic_store_n(&fail, 1, __ATOMIC_RELAXED);
  }
  gg_graph *u = fail ? NULL : (gg_graph *)calloc(1, sizeof(gg_graph));
  if (u) {
    vo_out[0] = 0;
    for (int64_t k = 0; k < G; ++k) {
      vo_out[k + 1] = vo_out[k] + parts[k]->n;
      eo[k + 1] = eo[k] + parts[k]->nnz;
    }
    u->n = vo_out[G];
    u->nnz = eo[G];
    u->off = (int64_t *)malloc(((size_t)u->n + 1) * sizeof(int64_t));
    u->col = (int32_t *)malloc((size_t)(u->nnz > 0 ? u->nnz : 1) * sizeof(int32_t));
    if (!u->off || !u->col) { free(u->off); free(u->col); free(u); u = NULL; }
  }
  if (u) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < G; ++k) {
      const gg_graph *p = parts[k];
      const int64_t v0 = vo_out[k], e0 = eo[k];
      for (int64_t i = 0; i < p->n; ++i) u->off[v0 + i] = p->off[i] + e0;
      for (int64_t e = 0; e < p->nnz; ++e) u->col[e0 + e] = (int32_t)(p->col[e] + v0);
    }
    u->off[u->n] = u->nnz;
  }
  for (int64_t k = 0; k < G; ++k) gg_free(parts[k]);
  free(parts);
  free(eo);
  return u;
}

/* side x side 4-neighbour grid plus round(frac * grid_edges) uniform random
 * long-range pairs; weights uniform integers in [wlo, whi] per unordered pair. */
gg_graph *gg_grid(int64_t side, double frac, uint64_t seed, int wlo, int whi) {
  if (side < 2) return NULL;
  int64_t n = side * side;
  int64_t ng = 2 * side * (side - 1);
  int64_t nl = (int64_t)llround(frac * (double)ng);
  int64_t np = ng + nl;
  uint32_t *pu = (uint32_t *)malloc((size_t)np * sizeof(uint32_t));
  uint32_t *pv = (uint32_t *)malloc((size_t)np * sizeof(uint32_t));
  if (!pu || !pv) { free(pu); free(pv); return NULL; }
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < side; ++r) {
    for (int64_t c = 0; c < side; ++c) {
      int64_t id = r * side + c;
      /* horizontal edges are numbered r*(side-1)+c, vertical ones after them */
      if (c + 1 < side) {
        int64_t k = r * (side - 1) + c;
        pu[k] = (uint32_t)id; pv[k] = (uint32_t)(id + 1);
      }
      if (r + 1 < side) {
        int64_t k = side * (side - 1) + r * side + c;
        pu[k] = (uint32_t)id; pv[k] = (uint32_t)(id + side);
      }
    }
  }
  const uint64_t s = sm64(seed, 0x4C4F4E47ULL); /* "LONG" sub-stream */
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < nl; ++k) {
    pu[ng + k] = (uint32_t)(sm64(s, 2 * (uint64_t)k) % (uint64_t)n);
    pv[ng + k] = (uint32_t)(sm64(s, 2 * (uint64_t)k + 1) % (uint64_t)n);
  }
  weight_rule wr = {sm64(seed, 0x57474854ULL), wlo, whi};
  return build_csr(n, np, pu, pv, (wlo == 1 && whi == 1) ? NULL : &wr);
}

/* Generic: CSR from a caller-supplied undirected pair list (copied). */
gg_graph *gg_from_pairs(int64_t n, int64_t np, const int64_t *u, const int64_t *v) {
  uint32_t *pu = (uint32_t *)malloc((size_t)(np > 0 ? np : 1) * sizeof(uint32_t));
  uint32_t *pv = (uint32_t *)malloc((size_t)(np > 0 ? np : 1) * sizeof(uint32_t));
  if (!pu || !pv) { free(pu); free(pv); return NULL; }
  for (int64_t k = 0; k < np; ++k) {
    if (u[k] < 0 || u[k] >= n || v[k] < 0 || v[k] >= n) { free(pu); free(pv); return NULL; }
    pu[k] = (uint32_t)u[k];
    pv[k] = (uint32_t)v[k];
  }
  return build_csr(n, np, pu, pv, NULL);
}

int gg_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
