/*
 * Seeded synthetic graph generators (input side only).
 *
 * This module produces undirected edge lists for tests, the benchmark and the
 * oracle's stored digests.  It holds none of the truss-decomposition arithmetic:
 * no supports, no orientation, no peeling.  Both the CPU oracle and the GPU
 * library consume its output; neither is used here.
 *
 * Randomness: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) used in counter mode: draw(seed, stream, ctr)
 * is the ctr-th output of the SplitMix64 sequence whose starting state is a mix
 * of (seed, stream).  Probabilities are compared as 32-bit integer thresholds.
 * The few real-valued steps (Chung-Lu weights, alias table, log-uniform sizes,
 * Poisson arrivals) use only IEEE +,-,*,/ and exact scalings (ldexp/frexp) in a
 * fixed order; logarithm and exponential are series written here, so results
 * are bit-identical on x86-64 and aarch64 when compiled with
 * -ffp-contract=off (no fused multiply-add).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Start state of stream `stream` under `seed`. */
static inline uint64_t sm_key(uint64_t seed, uint64_t stream) {
  return sm_mix(sm_mix(seed + GOLDEN) ^ (stream * GOLDEN + 0x632BE59BD9B4E019ULL));
}

/* ctr-th SplitMix64 output from start state `key` (state advances by GOLDEN). */
static inline uint64_t sm_at(uint64_t key, uint64_t ctr) {
  return sm_mix(key + (ctr + 1) * GOLDEN);
}

uint64_t gg_splitmix64(uint64_t x) { return sm_mix(x + GOLDEN); }

uint64_t gg_draw(uint64_t seed, uint64_t stream, uint64_t ctr) {
  return sm_at(sm_key(seed, stream), ctr);
}

/* Uniform integer in [0, n) by 64x64->128 multiply-shift. */
static inline uint64_t below(uint64_t r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
}

/* ---------------------------------------------------------------- maths --- */
/* Natural logarithm for x > 0: x = f * 2^e with f in [sqrt(1/2), sqrt(2)),
 * ln f = 2 atanh(s), s = (f-1)/(f+1), by its odd power series. */
static double gg_log(double x) {
  int e;
  double f = frexp(x, &e); /* f in [0.5, 1) */
  if (f < 0.70710678118654752) { f = f * 2.0; e -= 1; }
  double s = (f - 1.0) / (f + 1.0);
  double s2 = s * s, term = s, acc = 0.0;
  for (int j = 1; j <= 41; j += 2) { acc = acc + term / (double)j; term = term * s2; }
  return 2.0 * acc + (double)e * 0.69314718055994530942;
}

/* Exponential: t = k ln2 + r, |r| <= ln2/2, exp(r) by its Taylor series. */
static double gg_exp(double t) {
  double kf = floor(t / 0.69314718055994530942 + 0.5);
  double r = t - kf * 0.69314718055994530942;
  double term = 1.0, acc = 1.0;
  for (int j = 1; j <= 24; j++) { term = term * r / (double)j; acc = acc + term; }
  return ldexp(acc, (int)kf);
}

double gg_log_public(double x) { return gg_log(x); }
double gg_exp_public(double x) { return gg_exp(x); }

/* Uniform double in [0,1) with 53 random bits. */
static inline double unit53(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------ hash set --- */
typedef struct { uint64_t *slot; uint64_t mask; } pairset;

static int ps_init(pairset *s, int64_t expect) {
  uint64_t cap = 16;
  while (cap < (uint64_t)expect * 2 + 16) cap <<= 1;
  s->slot = (uint64_t *)calloc(cap, sizeof(uint64_t));
  s->mask = cap - 1;
  return s->slot ? 0 : -1;
}
static void ps_free(pairset *s) { free(s->slot); s->slot = 0; }

/* Insert undirected pair {u,v} (u != v); returns 1 if it was new. */
static int ps_insert(pairset *s, uint32_t u, uint32_t v) {
  uint32_t a = u < v ? u : v, b = u < v ? v : u;
  uint64_t key = (((uint64_t)a << 32) | b) + 1; /* never 0 */
  uint64_t h = sm_mix(key) & s->mask;
  for (;;) {
    uint64_t cur = s->slot[h];
    if (cur == 0) { s->slot[h] = key; return 1; }
    if (cur == key) return 0;
    h = (h + 1) & s->mask;
  }
}

/* ----------------------------------------------------------- generators --- */
/* Erdos-Renyi G(n, m): the first m distinct non-loop unordered pairs of a
 * stream of uniform ordered pairs.  Rows keep the sampled orientation.
 * Returns the number of rows written (m, or fewer if max_draws ran out). */
int64_t gg_er(int64_t n, int64_t m, uint64_t seed, uint64_t stream,
              int32_t *src, int32_t *dst, int64_t max_draws) {
  if (n < 2 || m <= 0) return 0;
  pairset s;
  if (ps_init(&s, m)) return -1;
  uint64_t key = sm_key(seed, stream);
  int64_t k = 0;
  for (int64_t c = 0; k < m && c < max_draws; c++) {
    uint64_t r = sm_at(key, (uint64_t)c);
    uint32_t u = (uint32_t)below(r, (uint64_t)n);
    uint32_t v = (uint32_t)below(sm_mix(r ^ 0xD6E8FEB86659FD93ULL), (uint64_t)n);
    if (u == v) continue;
    if (!ps_insert(&s, u, v)) continue;
    src[k] = (int32_t)u; dst[k] = (int32_t)v; k++;
  }
  ps_free(&s);
  return k;
}

/* One R-MAT sample: `scale` levels, each picking a quadrant with 32-bit
 * thresholds t1 < t2 < t3 (a, a+b, a+b+c of 2^32).  Two levels per draw. */
static inline void rmat_one(uint64_t key, uint64_t i, int scale, uint32_t t1, uint32_t t2,
                            uint32_t t3, uint32_t *pu, uint32_t *pv) {
  uint32_t u = 0, v = 0;
  uint64_t r = 0;
  for (int l = 0; l < scale; l++) {
    uint32_t x;
    if ((l & 1) == 0) { r = sm_at(key, i * 32 + (uint64_t)(l >> 1)); x = (uint32_t)(r >> 32); }
    else x = (uint32_t)r;
    uint32_t bu, bv;
    if (x < t1) { bu = 0; bv = 0; }
    else if (x < t2) { bu = 0; bv = 1; }
    else if (x < t3) { bu = 1; bv = 0; }
    else { bu = 1; bv = 1; }
    u = (u << 1) | bu; v = (v << 1) | bv;
  }
  *pu = u; *pv = v;
}

/* R-MAT raw samples: exactly `ns` rows, duplicates and self-loops kept. */
void gg_rmat_raw(int scale, int64_t ns, uint32_t t1, uint32_t t2, uint32_t t3, uint64_t seed,
                 uint64_t stream, int32_t *src, int32_t *dst) {
  uint64_t key = sm_key(seed, stream);
  for (int64_t i = 0; i < ns; i++) {
    uint32_t u, v;
    rmat_one(key, (uint64_t)i, scale, t1, t2, t3, &u, &v);
    src[i] = (int32_t)u; dst[i] = (int32_t)v;
  }
}

/* R-MAT, first m distinct non-loop pairs (at most max_draws samples). */
int64_t gg_rmat_distinct(int scale, int64_t m, uint32_t t1, uint32_t t2, uint32_t t3,
                         uint64_t seed, uint64_t stream, int32_t *src, int32_t *dst,
                         int64_t max_draws) {
  pairset s;
  if (ps_init(&s, m)) return -1;
  uint64_t key = sm_key(seed, stream);
  int64_t k = 0;
  for (int64_t i = 0; k < m && i < max_draws; i++) {
    uint32_t u, v;
    rmat_one(key, (uint64_t)i, scale, t1, t2, t3, &u, &v);
    if (u == v) continue;
    if (!ps_insert(&s, u, v)) continue;
    src[k] = (int32_t)u; dst[k] = (int32_t)v; k++;
  }
  ps_free(&s);
  return k;
}

/* Seeded permutation of 0..n-1 (Fisher-Yates, one draw per swap). */
void gg_permutation(int64_t n, uint64_t seed, uint64_t stream, int32_t *out) {
  uint64_t key = sm_key(seed, stream);
  for (int64_t i = 0; i < n; i++) out[i] = (int32_t)i;
  for (int64_t i = n - 1; i > 0; i--) {
    int64_t j = (int64_t)below(sm_at(key, (uint64_t)(n - 1 - i)), (uint64_t)(i + 1));
    int32_t t = out[i]; out[i] = out[j]; out[j] = t;
  }
}

/* Append the edges of cliques on consecutive slices of `verts` (sizes given)
 * to rows [m_in, ...), skipping pairs already present among the first m_in
 * rows or earlier cliques.  Returns the new row count. */
int64_t gg_add_cliques(int64_t m_in, int32_t *src, int32_t *dst, const int32_t *verts,
                       int nclq, const int32_t *sizes) {
  int64_t extra = 0;
  for (int c = 0; c < nclq; c++) extra += (int64_t)sizes[c] * (sizes[c] - 1) / 2;
  pairset s;
  if (ps_init(&s, m_in + extra)) return -1;
  for (int64_t i = 0; i < m_in; i++) ps_insert(&s, (uint32_t)src[i], (uint32_t)dst[i]);
  int64_t k = m_in, base = 0;
  for (int c = 0; c < nclq; c++) {
    for (int a = 0; a < sizes[c]; a++)
      for (int b = a + 1; b < sizes[c]; b++) {
        uint32_t u = (uint32_t)verts[base + a], v = (uint32_t)verts[base + b];
        if (!ps_insert(&s, u, v)) continue;
        src[k] = (int32_t)u; dst[k] = (int32_t)v; k++;
      }
    base += sizes[c];
  }
  ps_free(&s);
  return k;
}

/* ------------------------------------------------------------ Chung-Lu --- */
/* Expected-degree weights w_i = min(c (i+1)^(-1/(gamma-1)), cap), with c set by
 * bisection so that the mean weight is `mean`.  Writes w[n]; returns c. */
double gg_chung_lu_weights(int64_t n, double mean, double cap, double gamma, double *w) {
  double beta = 1.0 / (gamma - 1.0);
  for (int64_t i = 0; i < n; i++) w[i] = gg_exp(-beta * gg_log((double)(i + 1)));
  double lo = 0.0, hi = mean * (double)n + cap;
  for (int it = 0; it < 200; it++) {
    double c = 0.5 * (lo + hi);
    double sum = 0.0;
    for (int64_t i = 0; i < n; i++) { double x = c * w[i]; sum = sum + (x < cap ? x : cap); }
    if (sum / (double)n < mean) lo = c; else hi = c;
    if (hi - lo <= lo * 1e-15) break;
  }
  double c = 0.5 * (lo + hi);
  for (int64_t i = 0; i < n; i++) { double x = c * w[i]; w[i] = x < cap ? x : cap; }
  return c;
}

/* Walker/Vose alias table over weights w[n]: thr[i] in [0, 2^32] (as uint64),
 * sample i with probability thr[i]/2^32, else alias[i]. */
int gg_alias_build(int64_t n, const double *w, uint64_t *thr, int32_t *alias) {
  double W = 0.0;
  for (int64_t i = 0; i < n; i++) W = W + w[i];
  double *p = (double *)malloc(sizeof(double) * (size_t)n);
  int32_t *sm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  int32_t *lg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
  if (!p || !sm || !lg) { free(p); free(sm); free(lg); return -1; }
  int64_t ns = 0, nl = 0;
  for (int64_t i = 0; i < n; i++) {
    p[i] = w[i] * (double)n / W;
    if (p[i] < 1.0) sm[ns++] = (int32_t)i; else lg[nl++] = (int32_t)i;
    alias[i] = (int32_t)i;
  }
  while (ns > 0 && nl > 0) {
    int32_t s = sm[--ns], l = lg[--nl];
    thr[s] = (uint64_t)(p[s] * 4294967296.0);
    alias[s] = l;
    p[l] = (p[l] + p[s]) - 1.0;
    if (p[l] < 1.0) sm[ns++] = l; else lg[nl++] = l;
  }
  while (nl > 0) { int32_t l = lg[--nl]; thr[l] = 4294967296ULL; }
  while (ns > 0) { int32_t s = sm[--ns]; thr[s] = 4294967296ULL; }
  free(p); free(sm); free(lg);
  return 0;
}

static inline uint32_t alias_pick(uint64_t r, int64_t n, const uint64_t *thr, const int32_t *alias) {
  uint64_t i = below(r, (uint64_t)n);
  uint64_t lo = r & 0xFFFFFFFFULL;
  return lo < thr[i] ? (uint32_t)i : (uint32_t)alias[i];
}

/* Chung-Lu: first m distinct non-loop pairs, each endpoint drawn i.i.d.
 * proportional to the weights (alias table).  Returns rows written. */
int64_t gg_chung_lu(int64_t n, int64_t m, const uint64_t *thr, const int32_t *alias,
                    uint64_t seed, uint64_t stream, int32_t *src, int32_t *dst,
                    int64_t max_draws) {
  pairset s;
  if (ps_init(&s, m)) return -1;
  uint64_t key = sm_key(seed, stream);
  int64_t k = 0;
  for (int64_t c = 0; k < m && c < max_draws; c++) {
    uint32_t u = alias_pick(sm_at(key, 2 * (uint64_t)c), n, thr, alias);
    uint32_t v = alias_pick(sm_at(key, 2 * (uint64_t)c + 1), n, thr, alias);
    if (u == v) continue;
    if (!ps_insert(&s, u, v)) continue;
    src[k] = (int32_t)u; dst[k] = (int32_t)v; k++;
  }
  ps_free(&s);
  return k;
}

/* ----------------------------------------------------- batch and serve --- */
/* Parameters of graph g of the batched workload.
 * type 0: ER, 1: R-MAT, 2: ER plus one planted clique.  Edge target m is
 * log-uniform in [64, 65536]. */
void gg_batch_spec(int64_t g, uint64_t base, int32_t *type, int64_t *n, int64_t *m,
                   uint64_t *seed, int32_t *clique) {
  uint64_t sd = gg_splitmix64(base ^ (uint64_t)g);
  *seed = sd;
  *type = (int32_t)(g % 3);
  double u = unit53(gg_draw(sd, 100, 0));
  double lm = gg_log(64.0) + u * (gg_log(65536.0) - gg_log(64.0));
  int64_t mm = (int64_t)floor(gg_exp(lm) + 0.5);
  if (mm < 64) mm = 64;
  if (mm > 65536) mm = 65536;
  *m = mm;
  *clique = 0;
  if (*type == 1) {
    int sc = 4;
    while (((int64_t)1 << sc) < (mm + 7) / 8) sc++; /* 2^sc >= ceil(m/8) */
    *n = (int64_t)1 << sc;
  } else {
    int64_t nn = (mm + 3) / 4;
    if (nn < 16) nn = 16;
    if (*type == 2) {
      int32_t s = 4 + (int32_t)below(gg_draw(sd, 101, 0), 37); /* U{4..40} */
      *clique = s;
      if (nn < s) nn = s;
    }
    *n = nn;
  }
}

/* Serve request j: arrival time (s) accumulated from exponential gaps at rate
 * lambda, and edge target log-uniform in [mlo, mhi]. */
void gg_serve_schedule(int64_t count, double lambda, double mlo, double mhi, uint64_t seed,
                       double *t_arrive, int64_t *m) {
  double t = 0.0;
  for (int64_t j = 0; j < count; j++) {
    double u = unit53(gg_draw(seed, 200, (uint64_t)j));
    t = t + (-gg_log(1.0 - u)) / lambda;
    t_arrive[j] = t;
    double v = unit53(gg_draw(seed, 201, (uint64_t)j));
    double lm = gg_log(mlo) + v * (gg_log(mhi) - gg_log(mlo));
    m[j] = (int64_t)floor(gg_exp(lm) + 0.5);
  }
}

/* ------------------------------------------- first-m-distinct by sorting --- */
/* Same rows as gg_chung_lu (the first m distinct non-loop pairs of the
 * sample stream, in sample order), found by sorting instead of a hash set:
 * draw S samples, sort (pair key, sample index) with a stable LSD radix sort,
 * keep the first index of every key, then emit the first m kept samples in
 * sample order.  If S samples hold fewer than m distinct pairs, S grows. */
static void radix_sort_u64_idx(uint64_t *key, uint32_t *idx, uint64_t *tk, uint32_t *ti,
                               int64_t n, int bits) {
  enum { R = 11 };
  static int64_t cnt[1 << R];
  uint64_t *k0 = key, *k1 = tk;
  uint32_t *i0 = idx, *i1 = ti;
  const uint64_t mask = (1ull << R) - 1;
  for (int shift = 0; shift < bits; shift += R) {
    memset(cnt, 0, sizeof(cnt));
    for (int64_t i = 0; i < n; i++) cnt[(k0[i] >> shift) & mask]++;
    int64_t sum = 0;
    for (int b = 0; b < (1 << R); b++) {
      const int64_t c = cnt[b];
      cnt[b] = sum;
      sum += c;
    }
    for (int64_t i = 0; i < n; i++) {
      const int64_t p = cnt[(k0[i] >> shift) & mask]++;
      k1[p] = k0[i];
      i1[p] = i0[i];
    }
    uint64_t *tkp = k0; k0 = k1; k1 = tkp;   /* the sorted data is now in k0/i0 */
    uint32_t *tip = i0; i0 = i1; i1 = tip;
  }
  if (k0 != key) {
    memcpy(key, k0, sizeof(uint64_t) * (size_t)n);
    memcpy(idx, i0, sizeof(uint32_t) * (size_t)n);
  }
}

int64_t gg_chung_lu_sorted(int64_t n, int64_t m, const uint64_t *thr, const int32_t *alias,
                           uint64_t seed, uint64_t stream, int32_t *src, int32_t *dst) {
  uint64_t key0 = sm_key(seed, stream);
  int bits = 1;
  while (bits < 64 && ((uint64_t)1 << bits) < (uint64_t)n) bits++;
  int64_t S = m + m / 16 + 1024;
  for (;;) {
    if (S > 0xFFFFFFFFll) return -1;
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)S);
    uint64_t *tk = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)S);
    uint32_t *idx = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)S);
    uint32_t *ti = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)S);
    unsigned char *first = (unsigned char *)calloc((size_t)S, 1);
    if (!key || !tk || !idx || !ti || !first) {
      free(key); free(tk); free(idx); free(ti); free(first);
      return -1;
    }
    const uint64_t loop = ~0ull;
    for (int64_t c = 0; c < S; c++) {
      uint32_t u = alias_pick(sm_at(key0, 2 * (uint64_t)c), n, thr, alias);
      uint32_t v = alias_pick(sm_at(key0, 2 * (uint64_t)c + 1), n, thr, alias);
      key[c] = u == v ? loop : (((uint64_t)(u < v ? u : v) << bits) | (u < v ? v : u));
      idx[c] = (uint32_t)c;
    }
    radix_sort_u64_idx(key, idx, tk, ti, S, 64);
    int64_t distinct = 0;
    for (int64_t i = 0; i < S; i++) {
      if (key[i] == loop) continue;
      if (i == 0 || key[i] != key[i - 1]) { first[idx[i]] = 1; distinct++; }
    }
    if (distinct >= m) {
      int64_t k = 0;
      for (int64_t c = 0; c < S && k < m; c++) {
        if (!first[c]) continue;
        src[k] = (int32_t)alias_pick(sm_at(key0, 2 * (uint64_t)c), n, thr, alias);
        dst[k] = (int32_t)alias_pick(sm_at(key0, 2 * (uint64_t)c + 1), n, thr, alias);
        k++;
      }
      free(key); free(tk); free(idx); free(ti); free(first);
      return k;
    }
    free(key); free(tk); free(idx); free(ti); free(first);
    S = S + S / 2;
  }
}
