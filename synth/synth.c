/*
 * Seeded synthetic transaction databases (shared input generator).
 *
 * This module produces the synthetic inputs that stand in for the paper's
 * 20M / Tornado20M workloads (Section 5.1, Table 1). It holds none of the
 * mining method's arithmetic: it only draws random transactions and returns
 * them as CSR item lists (row_ptr[n+1], items[nnz]), each row sorted
 * ascending with no duplicates. Packing into bitmaps, counting and the
 * lattice live on each side (oracle and CUDA library) separately.
 *
 * Determinism: every random draw comes from a counter-based splitmix64
 * stream keyed by (seed, stream id, row), and all floating point is basic
 * IEEE arithmetic (own exp/log below, compiled with -ffp-contract=off), so
 * the same seed gives the same database on x86-64 and AArch64.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- RNG */
typedef struct { uint64_t s; } rng_t;

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static rng_t rng_make(uint64_t seed, uint64_t stream, uint64_t row) {
  rng_t r;
  r.s = mix64(seed ^ mix64(stream * 0x9E3779B97F4A7C15ULL + 0x632BE59BD9B4E019ULL) ^
              mix64(row + 0xD1B54A32D192ED03ULL));
  return r;
}
static uint64_t rng_next(rng_t *r) {
  r->s += 0x9E3779B97F4A7C15ULL;
  return mix64(r->s);
}
/* uniform in [0,1) with 53 random bits */
static double rng_unif(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, k) (multiply-shift; bias < 2^-32) */
static uint32_t rng_below(rng_t *r, uint32_t k) {
  return (uint32_t)(((rng_next(r) >> 32) * (uint64_t)k) >> 32);
}

/* ------------------------------------------- elementary functions
 * Written from the series definitions with basic operations only, so the
 * results do not depend on the platform's libm. */
static const double LN2 = 0.6931471805599453094;

static double d_ldexp(double x, int e) {
  while (e > 0) { x *= 2.0; --e; }
  while (e < 0) { x *= 0.5; ++e; }
  return x;
}
/* exp(x) = 2^k * exp(r), |r| <= ln2/2, Taylor series for exp(r) */
static double d_exp(double x) {
  if (x < -700.0) return 0.0;
  if (x > 700.0) x = 700.0;
  int k = (int)(x / LN2 + (x >= 0 ? 0.5 : -0.5));
  double r = x - (double)k * LN2;
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 30; ++i) { term = term * r / (double)i; sum += term; }
  return d_ldexp(sum, k);
}
/* log(x) for x > 0: x = 2^e * f, f in [1,2); log f = 2 atanh((f-1)/(f+1)) */
static double d_log(double x) {
  int e = 0;
  while (x >= 2.0) { x *= 0.5; ++e; }
  while (x < 1.0) { x *= 2.0; --e; }
  double y = (x - 1.0) / (x + 1.0), y2 = y * y, term = y, sum = 0.0;
  for (int i = 1; i < 80; i += 2) { sum += term / (double)i; term *= y2; }
  return 2.0 * sum + (double)e * LN2;
}
static double d_pow(double a, double b) { return d_exp(b * d_log(a)); }

/* Poisson(lambda) by Knuth's product-of-uniforms method (lambda <= ~60) */
static uint32_t rng_poisson(rng_t *r, double lambda) {
  double L = d_exp(-lambda), p = 1.0;
  uint32_t k = 0;
  do { ++k; p *= rng_unif(r); } while (p > L && k < 100000);
  return k - 1;
}
/* Exp(1) */
static double rng_exp1(rng_t *r) {
  double u = rng_unif(r);
  return -d_log(1.0 - u);
}

/* ------------------------------------------------------ output buffer */
typedef struct { uint32_t *v; uint64_t n, cap; } vec_u32;
static int vpush(vec_u32 *a, uint32_t x) {
  if (a->n == a->cap) {
    uint64_t nc = a->cap ? a->cap * 2 : 1024;
    uint32_t *nv = (uint32_t *)realloc(a->v, nc * sizeof(uint32_t));
    if (!nv) return -1;
    a->v = nv; a->cap = nc;
  }
  a->v[a->n++] = x;
  return 0;
}

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return x < y ? -1 : x > y;
}

/* A row under construction: membership bitmap (scratch) + item list. */
typedef struct { uint8_t *in; uint32_t *list; uint32_t len; } row_t;
static void row_add(row_t *w, uint32_t item) {
  if (!w->in[item]) { w->in[item] = 1; w->list[w->len++] = item; }
}
static int row_flush(row_t *w, vec_u32 *out) {
  qsort(w->list, w->len, sizeof(uint32_t), cmp_u32);
  for (uint32_t i = 0; i < w->len; ++i) {
    w->in[w->list[i]] = 0;
    if (vpush(out, w->list[i])) return -1;
  }
  w->len = 0;
  return 0;
}

/* Pattern pool: lengths, items (CSR) and cumulative weights. */
typedef struct { uint32_t np; uint32_t *off; uint32_t *items; double *cum; } pool_t;

static void pool_free(pool_t *p) { free(p->off); free(p->items); free(p->cum); }

/* Build np patterns over m items. Length Poisson(len_mean) clipped to
 * [1, m]; the first floor(carry*len) items are drawn from the previous
 * pattern, the rest uniformly (all distinct within a pattern); weights are
 * Exp(1), normalised into a cumulative table. */
static int pool_build(pool_t *p, uint64_t seed, uint32_t np, uint32_t m, double len_mean,
                      double carry) {
  memset(p, 0, sizeof(*p));
  p->np = np;
  p->off = (uint32_t *)calloc((size_t)np + 1, sizeof(uint32_t));
  p->cum = (double *)calloc(np ? np : 1, sizeof(double));
  uint8_t *in = (uint8_t *)calloc(m, 1);
  vec_u32 items = {0, 0, 0};
  if (!p->off || !p->cum || !in) { free(in); pool_free(p); return -1; }
  double wsum = 0.0;
  for (uint32_t j = 0; j < np; ++j) {
    rng_t r = rng_make(seed, 1, j);
    uint32_t len = rng_poisson(&r, len_mean);
    if (len < 1) len = 1;
    if (len > m) len = m;
    uint32_t start = (uint32_t)items.n, got = 0;
    if (j > 0 && carry > 0.0) {
      uint32_t ps = p->off[j - 1], plen = p->off[j] - ps;
      uint32_t want = (uint32_t)(carry * (double)len);
      if (want > plen) want = plen;
      for (uint32_t tries = 0; got < want && tries < 64 * (want + 1); ++tries) {
        uint32_t it = items.v[ps + rng_below(&r, plen)];
        if (!in[it]) { in[it] = 1; if (vpush(&items, it)) goto fail; ++got; }
      }
    }
    while (got < len) {
      uint32_t it = rng_below(&r, m);
      if (!in[it]) { in[it] = 1; if (vpush(&items, it)) goto fail; ++got; }
    }
    for (uint32_t i = start; i < items.n; ++i) in[items.v[i]] = 0;
    p->off[j + 1] = (uint32_t)items.n;
    wsum += rng_exp1(&r);
    p->cum[j] = wsum;
  }
  for (uint32_t j = 0; j < np; ++j) p->cum[j] /= wsum;
  p->items = items.v;
  free(in);
  return 0;
fail:
  free(in); free(items.v); pool_free(p);
  return -1;
}

static uint32_t pool_draw(const pool_t *p, rng_t *r) {
  double u = rng_unif(r);
  uint32_t lo = 0, hi = p->np - 1;
  while (lo < hi) {
    uint32_t mid = (lo + hi) / 2;
    if (p->cum[mid] > u) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/*
 * Planted-pattern database.
 *   n, m            transactions, items
 *   n_patterns      pool size; pattern length Poisson(pat_len_mean) >= 1
 *   carry           fraction of a pattern's items carried over from the
 *                   previous pattern
 *   tx_len_mean     transaction length target ~ Poisson(tx_len_mean)
 *   keep_p          each item of a drawn pattern is kept with this prob.
 *   noise_frac      Binomial(target, noise_frac) uniform noise items
 * A row is filled with noise first, then by weighted pattern draws until it
 * reaches its target length (a draw that would overshoot is truncated); at
 * most 4*target+16 draws are made, so a row may end shorter.
 */
int synth_planted(uint64_t seed, uint64_t n, uint32_t m, uint32_t n_patterns,
                  double pat_len_mean, double carry, double tx_len_mean, double keep_p,
                  double noise_frac, uint64_t *row_ptr, uint32_t **items_out, uint64_t *nnz_out) {
  *items_out = NULL; *nnz_out = 0;
  if (m == 0 || n_patterns == 0) return -2;
  pool_t pool;
  if (pool_build(&pool, seed, n_patterns, m, pat_len_mean, carry)) return -1;
  row_t w;
  w.in = (uint8_t *)calloc(m, 1);
  w.list = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
  w.len = 0;
  vec_u32 out = {0, 0, 0};
  if (!w.in || !w.list) goto fail;
  row_ptr[0] = 0;
  for (uint64_t t = 0; t < n; ++t) {
    rng_t r = rng_make(seed, 2, t);
    uint32_t target = rng_poisson(&r, tx_len_mean);
    if (target > m) target = m;
    uint32_t noise = 0;
    for (uint32_t i = 0; i < target; ++i) noise += rng_unif(&r) < noise_frac;
    for (uint32_t i = 0; i < noise; ++i) row_add(&w, rng_below(&r, m));
    for (uint32_t d = 0; d < 4 * target + 16 && w.len < target; ++d) {
      uint32_t j = pool_draw(&pool, &r);
      for (uint32_t q = pool.off[j]; q < pool.off[j + 1] && w.len < target; ++q)
        if (rng_unif(&r) < keep_p) row_add(&w, pool.items[q]);
    }
    if (row_flush(&w, &out)) goto fail;
    row_ptr[t + 1] = out.n;
  }
  free(w.in); free(w.list); pool_free(&pool);
  *items_out = out.v; *nnz_out = out.n;
  return 0;
fail:
  free(w.in); free(w.list); free(out.v); pool_free(&pool);
  return -1;
}

/*
 * Dense database: independent "noise" items with Zipf(zipf_s) popularity by
 * a seeded random rank, each item's inclusion probability capped at `cap`
 * and scaled so the expected noise count per row is noise_mean; plus
 * Poisson(draws_mean) weighted draws from a pool of n_patterns patterns of
 * Poisson(pat_len_mean) length, each item kept with keep_p.
 */
int synth_dense(uint64_t seed, uint64_t n, uint32_t m, double zipf_s, double noise_mean,
                double cap, uint32_t n_patterns, double pat_len_mean, double draws_mean,
                double keep_p, uint64_t *row_ptr, uint32_t **items_out, uint64_t *nnz_out,
                double *q_out /* m, may be NULL */) {
  *items_out = NULL; *nnz_out = 0;
  if (m == 0 || n_patterns == 0 || noise_mean >= cap * (double)m) return -2;
  double *q = (double *)malloc((size_t)m * sizeof(double));
  uint32_t *rank = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
  if (!q || !rank) { free(q); free(rank); return -1; }
  /* random rank permutation (Fisher-Yates) */
  {
    rng_t r = rng_make(seed, 3, 0);
    for (uint32_t i = 0; i < m; ++i) rank[i] = i;
    for (uint32_t i = m - 1; i > 0; --i) {
      uint32_t j = rng_below(&r, i + 1), tmp = rank[i];
      rank[i] = rank[j]; rank[j] = tmp;
    }
  }
  double *base = (double *)malloc((size_t)m * sizeof(double));
  if (!base) { free(q); free(rank); return -1; }
  for (uint32_t i = 0; i < m; ++i) base[i] = d_pow((double)(rank[i] + 1), -zipf_s);
  /* bisection on the scale c so that sum_i min(cap, c*base_i) = noise_mean */
  double lo = 0.0, hi = 1.0;
  for (;;) {
    double s = 0.0;
    for (uint32_t i = 0; i < m; ++i) { double v = hi * base[i]; s += v < cap ? v : cap; }
    if (s >= noise_mean || hi > 1e12) break;
    hi *= 2.0;
  }
  for (int it = 0; it < 200; ++it) {
    double c = 0.5 * (lo + hi), s = 0.0;
    for (uint32_t i = 0; i < m; ++i) { double v = c * base[i]; s += v < cap ? v : cap; }
    if (s > noise_mean) hi = c; else lo = c;
  }
  for (uint32_t i = 0; i < m; ++i) { double v = lo * base[i]; q[i] = v < cap ? v : cap; }
  free(base); free(rank);
  if (q_out) memcpy(q_out, q, (size_t)m * sizeof(double));

  pool_t pool;
  if (pool_build(&pool, seed, n_patterns, m, pat_len_mean, 0.0)) { free(q); return -1; }
  row_t w;
  w.in = (uint8_t *)calloc(m, 1);
  w.list = (uint32_t *)malloc((size_t)m * sizeof(uint32_t));
  w.len = 0;
  vec_u32 out = {0, 0, 0};
  if (!w.in || !w.list) goto fail;
  row_ptr[0] = 0;
  for (uint64_t t = 0; t < n; ++t) {
    rng_t r = rng_make(seed, 4, t);
    for (uint32_t i = 0; i < m; ++i)
      if (rng_unif(&r) < q[i]) row_add(&w, i);
    uint32_t draws = rng_poisson(&r, draws_mean);
    for (uint32_t d = 0; d < draws; ++d) {
      uint32_t j = pool_draw(&pool, &r);
      for (uint32_t x = pool.off[j]; x < pool.off[j + 1]; ++x)
        if (rng_unif(&r) < keep_p) row_add(&w, pool.items[x]);
    }
    if (row_flush(&w, &out)) goto fail;
    row_ptr[t + 1] = out.n;
  }
  free(w.in); free(w.list); pool_free(&pool); free(q);
  *items_out = out.v; *nnz_out = out.n;
  return 0;
fail:
  free(w.in); free(w.list); free(out.v); pool_free(&pool); free(q);
  return -1;
}

/* Uniform, log-uniform draws for the batched / served recipes: the i-th
 * value of stream `stream` under `seed`, in [0,1). */
double synth_uniform(uint64_t seed, uint64_t stream, uint64_t i) {
  rng_t r = rng_make(seed, 100 + stream, i);
  return rng_unif(&r);
}

void synth_free(void *p) { free(p); }
