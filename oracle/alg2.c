/*
 * CPU ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, single-threaded, slow-but-obvious truss decomposition following
 * Wang & Cheng, "Truss Decomposition in Massive Networks", Section 3.2,
 * Algorithm 2 ("improved truss decomposition"), with the supports of step 2
 * computed by the in-memory triangle counting algorithm the paper cites for
 * it (Section 3.2 and Theorem 1: the "forward" degree-ordered listing).
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may call this file.  It shares no code, header or table with the GPU
 * library and includes nothing from it.
 *
 * Definitions (Section 2): sup(e) is the number of triangles containing e
 * (Definition 1); the k-truss T_k is the largest subgraph whose edges each lie
 * in >= k-2 triangles inside it (Definition 2); phi(e) = max{k : e in T_k}.
 *
 * Readings where the paper leaves a choice (all result-neutral):
 *  - Step 9 decrements a partner edge only while its support is > k-2, so the
 *    bin-sorted array stays sorted behind the pointer; an edge already at
 *    <= k-2 is removed at this level either way.
 *  - "(v,w) in E_G" in step 8 means present and not yet removed; removed
 *    edges are those left of the pointer.
 *  - Ties for "the edge with the lowest support" follow bin order, which
 *    starts stable by edge id.
 *  - deg() in step 6 is the degree in the input graph; ties go to the smaller
 *    vertex id.
 *  - Output is per input row: support is sup(e, G) (Definition 1) and truss is
 *    phi(e); duplicate rows share their edge's values; self-loop rows get -1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* ---- edge hashtable (Section 3.2: membership test of step 8 by hashing) --- */
typedef struct {
  uint64_t *key; /* (a<<32|b)+1, 0 = empty */
  int32_t *val;  /* edge id */
  uint64_t mask;
  int shift;
} etable;

static uint64_t et_slot(const etable *t, uint64_t key) {
  return (key * 0x9E3779B97F4A7C15ULL) >> t->shift;
}

static int et_init(etable *t, int64_t m) {
  uint64_t cap = 16;
  int bits = 4;
  while (cap < (uint64_t)m * 2 + 16) { cap <<= 1; bits++; }
  t->key = (uint64_t *)calloc(cap, sizeof(uint64_t));
  t->val = (int32_t *)malloc(cap * sizeof(int32_t));
  t->mask = cap - 1;
  t->shift = 64 - bits;
  return (t->key && t->val) ? 0 : -1;
}

static void et_free(etable *t) { free(t->key); free(t->val); }

static void et_put(etable *t, int32_t a, int32_t b, int32_t e) {
  uint64_t key = (((uint64_t)(uint32_t)a << 32) | (uint32_t)b) + 1;
  uint64_t h = et_slot(t, key);
  while (t->key[h] != 0) h = (h + 1) & t->mask;
  t->key[h] = key;
  t->val[h] = e;
}

/* Edge id of {a,b}, or -1 if absent. */
static int32_t et_get(const etable *t, int32_t a, int32_t b) {
  if (a > b) { int32_t x = a; a = b; b = x; }
  uint64_t key = (((uint64_t)(uint32_t)a << 32) | (uint32_t)b) + 1;
  uint64_t h = et_slot(t, key);
  for (;;) {
    uint64_t k = t->key[h];
    if (k == key) return t->val[h];
    if (k == 0) return -1;
    h = (h + 1) & t->mask;
  }
}

/* ------------------------------------------------------------- graph --- */
typedef struct {
  int64_t n, m;
  int32_t *eu, *ev;  /* endpoints of edge e, eu < ev (lexicographic edge ids) */
  int64_t *off;      /* nb(v) = adj[off[v] .. off[v+1]), sorted by id */
  int32_t *adj;      /* neighbour ids */
  int32_t *adje;     /* edge id of (v, adj[j]) */
  int32_t *row2e;    /* input row -> edge id, -1 for self-loops */
  etable tab;
} graph;

static void g_free(graph *g) {
  free(g->eu); free(g->ev); free(g->off); free(g->adj); free(g->adje); free(g->row2e);
  et_free(&g->tab);
}

/* Simple graph from rows (Section 2: undirected, unweighted, simple).
 * Edge ids are positions in the sorted list of distinct pairs (min, max). */
static int g_build(graph *g, int64_t n, int64_t rows, const int32_t *src, const int32_t *dst) {
  memset(g, 0, sizeof(*g));
  g->n = n;
  for (int64_t r = 0; r < rows; r++)
    if (src[r] < 0 || src[r] >= n || dst[r] < 0 || dst[r] >= n) return OR_EINVAL;
  uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(rows > 0 ? rows : 1));
  if (!keys) return OR_ENOMEM;
  int64_t nk = 0;
  for (int64_t r = 0; r < rows; r++) {
    int32_t a = src[r], b = dst[r];
    if (a == b) continue;
    if (a > b) { int32_t x = a; a = b; b = x; }
    keys[nk++] = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
  }
  qsort(keys, (size_t)nk, sizeof(uint64_t), cmp_u64);
  int64_t m = 0;
  for (int64_t i = 0; i < nk; i++)
    if (i == 0 || keys[i] != keys[i - 1]) keys[m++] = keys[i];
  g->m = m;
  g->eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
  g->ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
  g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  g->adj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
  g->adje = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
  g->row2e = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rows + 1));
  if (!g->eu || !g->ev || !g->off || !g->adj || !g->adje || !g->row2e || et_init(&g->tab, m)) {
    free(keys);
    return OR_ENOMEM;
  }
  for (int64_t e = 0; e < m; e++) {
    g->eu[e] = (int32_t)(keys[e] >> 32);
    g->ev[e] = (int32_t)(keys[e] & 0xFFFFFFFFu);
    et_put(&g->tab, g->eu[e], g->ev[e], (int32_t)e);
  }
  free(keys);
  /* adjacency lists, sorted by neighbour id: edges arrive in (u,v) order, so
   * each list receives its smaller neighbours first, then its larger ones. */
  for (int64_t e = 0; e < m; e++) { g->off[g->eu[e] + 1]++; g->off[g->ev[e] + 1]++; }
  for (int64_t v = 0; v < n; v++) g->off[v + 1] += g->off[v];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!fill) return OR_ENOMEM;
  memcpy(fill, g->off, sizeof(int64_t) * (size_t)n);
  for (int64_t e = 0; e < m; e++) {
    int32_t a = g->eu[e], b = g->ev[e];
    g->adj[fill[a]] = b; g->adje[fill[a]++] = (int32_t)e;
    g->adj[fill[b]] = a; g->adje[fill[b]++] = (int32_t)e;
  }
  free(fill);
  for (int64_t r = 0; r < rows; r++)
    g->row2e[r] = (src[r] == dst[r]) ? -1 : et_get(&g->tab, src[r], dst[r]);
  return OR_OK;
}

static inline int64_t deg(const graph *g, int32_t v) { return g->off[v + 1] - g->off[v]; }

/* (deg(a), a) < (deg(b), b): the total order used by the forward algorithm. */
static inline int before(const graph *g, int32_t a, int32_t b) {
  int64_t da = deg(g, a), db = deg(g, b);
  return da < db || (da == db && a < b);
}

/* Step 2 of Algorithm 2: sup(e) for every edge by forward triangle listing.
 * Each triangle is listed once, from its first vertex u in the (deg, id)
 * order: v, w are later neighbours of u and w is a later neighbour of v.
 * Every listed triangle adds one to each of its three edges. Returns the
 * triangle count. */
static int64_t support_forward(const graph *g, int32_t *sup) {
  memset(sup, 0, sizeof(int32_t) * (size_t)g->m);
  /* later-neighbour lists A(v) = {w in nb(v) : v before w}, with edge ids */
  int64_t *aoff = (int64_t *)calloc((size_t)g->n + 1, sizeof(int64_t));
  int32_t *aw = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m + 1));
  int32_t *ae = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->m + 1));
  int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g->n + 1));
  for (int32_t v = 0; v < (int32_t)g->n; v++) {
    aoff[v + 1] = aoff[v];
    for (int64_t j = g->off[v]; j < g->off[v + 1]; j++)
      if (before(g, v, g->adj[j])) {
        aw[aoff[v + 1]] = g->adj[j];
        ae[aoff[v + 1]++] = g->adje[j];
      }
  }
  for (int64_t v = 0; v < g->n; v++) mark[v] = -1;
  int64_t tri = 0;
  for (int32_t u = 0; u < (int32_t)g->n; u++) {
    for (int64_t j = aoff[u]; j < aoff[u + 1]; j++) mark[aw[j]] = ae[j];  /* mark[w] = e_uw */
    for (int64_t j = aoff[u]; j < aoff[u + 1]; j++) {
      int32_t v = aw[j], e_uv = ae[j];
      for (int64_t q = aoff[v]; q < aoff[v + 1]; q++) {
        int32_t w = aw[q];
        if (mark[w] < 0) continue;
        sup[e_uv]++;
        sup[mark[w]]++;      /* e_uw */
        sup[ae[q]]++;        /* e_vw */
        tri++;
      }
    }
    for (int64_t j = aoff[u]; j < aoff[u + 1]; j++) mark[aw[j]] = -1;
  }
  free(aoff); free(aw); free(ae); free(mark);
  return tri;
}

/* Steps 3-16 of Algorithm 2 on supports s (consumed).  phi[e] receives the
 * truss number.  Returns k_max (2 for an edgeless graph with m = 0 -> 0). */
static int32_t peel_alg2(const graph *g, int32_t *s, int32_t *phi) {
  int64_t m = g->m;
  if (m == 0) return 0;
  int32_t smax = 0;
  for (int64_t e = 0; e < m; e++) if (s[e] > smax) smax = s[e];
  /* Step 3: bin sort, ascending support, stable by edge id. */
  int64_t *bin = (int64_t *)calloc((size_t)smax + 2, sizeof(int64_t));
  int32_t *A = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
  int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  unsigned char *dead = (unsigned char *)calloc((size_t)m, 1);
  for (int64_t e = 0; e < m; e++) bin[s[e] + 1]++;
  for (int32_t x = 0; x <= smax; x++) bin[x + 1] += bin[x];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)smax + 1));
  memcpy(fill, bin, sizeof(int64_t) * ((size_t)smax + 1));
  for (int64_t e = 0; e < m; e++) { pos[e] = fill[s[e]]; A[pos[e]] = (int32_t)e; fill[s[e]]++; }
  free(fill);

  int32_t k = 2, kmax = 2;
  int64_t i = 0;
  while (i < m) {
    /* Steps 4-12: remove lowest-support edges while sup <= k-2. */
    while (i < m && s[A[i]] <= k - 2) {
      int32_t e = A[i];
      int32_t u = g->eu[e], v = g->ev[e];
      if (!(deg(g, u) < deg(g, v) || (deg(g, u) == deg(g, v) && u < v))) {
        int32_t t = u; u = v; v = t;              /* step 6: deg(u) <= deg(v) */
      }
      for (int64_t j = g->off[u]; j < g->off[u + 1]; j++) { /* step 7 */
        int32_t w = g->adj[j];
        if (w == v) continue;
        int32_t e_uw = g->adje[j];
        if (dead[e_uw]) continue;
        int32_t e_vw = et_get(&g->tab, v, w);                  /* step 8 */
        if (e_vw < 0 || dead[e_vw]) continue;
        int32_t part[2] = {e_uw, e_vw};
        for (int p = 0; p < 2; p++) {                           /* steps 9-10 */
          int32_t x = part[p];
          int32_t sx = s[x];
          if (sx <= k - 2) continue;
          int64_t first = bin[sx];                /* move x to the front of its bin */
          int32_t y = A[first];
          int64_t px = pos[x];
          A[first] = x; pos[x] = first;
          A[px] = y; pos[y] = px;
          bin[sx]++;
          s[x] = sx - 1;
        }
      }
      phi[e] = k;                                               /* step 11 */
      dead[e] = 1;                                              /* step 12 */
      kmax = k;
      i++;
    }
    k++;                                                        /* step 14 */
  }
  free(bin); free(A); free(pos); free(dead);
  return kmax;
}

/* Public entry: per-row support and truss number (see header comment).
 * Returns 0, -1 (id out of range) or -2 (out of memory). */
int oracle_truss(int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
                 int32_t *support_out, int32_t *truss_out, int32_t *kmax_out,
                 int64_t *m_out, int64_t *tri_out) {
  graph g;
  int rc = g_build(&g, n, rows, src, dst);
  if (rc) { g_free(&g); return rc; }
  int32_t *sup = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.m + 1));
  int32_t *res = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.m + 1));
  int32_t *phi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.m + 1));
  if (!sup || !res || !phi) { free(sup); free(res); free(phi); g_free(&g); return OR_ENOMEM; }
  int64_t tri = support_forward(&g, sup);
  int32_t kmax = 0;
  if (truss_out) {
    memcpy(res, sup, sizeof(int32_t) * (size_t)g.m);
    kmax = peel_alg2(&g, res, phi);
  }
  for (int64_t r = 0; r < rows; r++) {
    int32_t e = g.row2e[r];
    if (support_out) support_out[r] = e < 0 ? -1 : sup[e];
    if (truss_out) truss_out[r] = e < 0 ? -1 : phi[e];
  }
  if (kmax_out) *kmax_out = kmax;
  if (m_out) *m_out = g.m;
  if (tri_out) *tri_out = tri;
  free(sup); free(res); free(phi);
  g_free(&g);
  return OR_OK;
}

/* Largest x such that at least x of the supports of w's incident edges,
 * leaving out edge `skip`, are >= x (the x_w of Procedure 6, Section 6.2),
 * by counting: cnt[x] = how many of those supports are >= x, for x <= deg. */
static int32_t x_excluding(const graph *g, const int32_t *sup, int32_t w, int32_t skip,
                           int64_t *cnt) {
  const int64_t d = deg(g, w);
  for (int64_t x = 0; x <= d; x++) cnt[x] = 0;
  for (int64_t j = g->off[w]; j < g->off[w + 1]; j++) {
    int32_t f = g->adje[j];
    if (f == skip) continue;
    int64_t s = sup[f] < d ? sup[f] : d;
    cnt[s]++;
  }
  /* suffix sums: cnt[x] = #{supports >= x} (capped supports keep this exact
   * for every x <= d) */
  for (int64_t x = d - 1; x >= 0; x--) cnt[x] += cnt[x + 1];
  int32_t best = 0;
  for (int64_t x = 0; x <= d; x++)
    if (cnt[x] >= x) best = (int32_t)x;
  return best;
}

/* Per-row psi(e) = min{sup(e), x_u, x_v} + 2 (Procedure 6 with the whole
 * graph as the neighbourhood subgraph) and sup(e); -1 for self-loop rows. */
int oracle_psi(int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
               int32_t *support_out, int32_t *psi_out) {
  graph g;
  int rc = g_build(&g, n, rows, src, dst);
  if (rc) { g_free(&g); return rc; }
  int64_t maxd = 0;
  for (int64_t v = 0; v < n; v++) if (deg(&g, v) > maxd) maxd = deg(&g, v);
  int32_t *sup = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.m + 1));
  int32_t *psi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.m + 1));
  int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxd + 2));
  if (!sup || !psi || !cnt) { free(sup); free(psi); free(cnt); g_free(&g); return OR_ENOMEM; }
  support_forward(&g, sup);
  for (int64_t e = 0; e < g.m; e++) {
    int32_t xu = x_excluding(&g, sup, g.eu[e], (int32_t)e, cnt);
    int32_t xv = x_excluding(&g, sup, g.ev[e], (int32_t)e, cnt);
    int32_t x = sup[e];
    if (xu < x) x = xu;
    if (xv < x) x = xv;
    psi[e] = x + 2;
  }
  for (int64_t r = 0; r < rows; r++) {
    int32_t e = g.row2e[r];
    if (support_out) support_out[r] = e < 0 ? -1 : sup[e];
    if (psi_out) psi_out[r] = e < 0 ? -1 : psi[e];
  }
  free(sup); free(psi); free(cnt);
  g_free(&g);
  return OR_OK;
}

/* Core number of every vertex (the largest k such that v lies in the k-core,
 * the largest subgraph of minimum degree >= k), by the bin-sorted degree
 * array that Section 3.2 borrows for its edge bins: vertices sit in an array
 * ordered by current degree with the start of each degree's block recorded;
 * the vertex at the front is removed with its current degree as its core
 * number, and each neighbour of larger current degree moves to the front of
 * its block, which then starts one later, and loses one degree.
 * core_out has n entries, indexed by vertex id; *kmax_out = max core. */
int oracle_core(int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
                int32_t *core_out, int32_t *kmax_out) {
  graph g;
  int rc = g_build(&g, n, rows, src, dst);
  if (rc) { g_free(&g); return rc; }
  int64_t maxd = 0;
  for (int64_t v = 0; v < n; v++) if (deg(&g, v) > maxd) maxd = deg(&g, v);
  int64_t *d = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t *start = (int64_t *)calloc((size_t)maxd + 2, sizeof(int64_t));
  int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int32_t *vert = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
  if (!d || !start || !pos || !vert) {
    free(d); free(start); free(pos); free(vert); g_free(&g);
    return OR_ENOMEM;
  }
  for (int64_t v = 0; v < n; v++) { d[v] = deg(&g, v); start[d[v] + 1]++; }
  for (int64_t k = 0; k <= maxd; k++) start[k + 1] += start[k];
  {
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxd + 1));
    if (!fill) { free(d); free(start); free(pos); free(vert); g_free(&g); return OR_ENOMEM; }
    for (int64_t k = 0; k <= maxd; k++) fill[k] = start[k];
    for (int64_t v = 0; v < n; v++) { pos[v] = fill[d[v]]++; vert[pos[v]] = (int32_t)v; }
    free(fill);
  }
  int32_t kmax = 0;
  for (int64_t i = 0; i < n; i++) {
    int32_t v = vert[i];
    core_out[v] = (int32_t)d[v];
    if (d[v] > kmax) kmax = (int32_t)d[v];
    for (int64_t j = g.off[v]; j < g.off[v + 1]; j++) {
      int32_t u = g.adj[j];
      if (d[u] > d[v]) {
        /* swap u with the first vertex of its block, shrink the block */
        int64_t du = d[u], pu = pos[u], pw = start[du];
        int32_t w = vert[pw];
        if (u != w) { vert[pu] = w; pos[w] = pu; vert[pw] = u; pos[u] = pw; }
        start[du]++;
        d[u]--;
      }
    }
  }
  if (kmax_out) *kmax_out = kmax;
  free(d); free(start); free(pos); free(vert);
  g_free(&g);
  return OR_OK;
}

/* Edge list in the oracle's canonical order (for tests): eu[e] < ev[e]. */
int oracle_edges(int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
                 int32_t *eu, int32_t *ev, int32_t *row2e, int64_t *m_out) {
  graph g;
  int rc = g_build(&g, n, rows, src, dst);
  if (rc) { g_free(&g); return rc; }
  if (eu) memcpy(eu, g.eu, sizeof(int32_t) * (size_t)g.m);
  if (ev) memcpy(ev, g.ev, sizeof(int32_t) * (size_t)g.m);
  if (row2e) memcpy(row2e, g.row2e, sizeof(int32_t) * (size_t)rows);
  *m_out = g.m;
  g_free(&g);
  return OR_OK;
}

/* Validity of a claimed decomposition phi over canonical edges (Definition
 * 2): every edge e must lie in >= phi(e)-2 triangles whose other two edges
 * have phi >= phi(e).  Also checks phi = 2 <=> sup = 0 and 2 <= phi <= sup+2.
 * Returns the number of violating edges (0 = valid). */
int64_t oracle_check_valid(int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
                           const int32_t *truss_rows, const int32_t *support_rows) {
  graph g;
  if (g_build(&g, n, rows, src, dst)) { g_free(&g); return -1; }
  int32_t *phi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.m + 1));
  int32_t *sup = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.m + 1));
  int32_t *in = (int32_t *)calloc((size_t)g.m + 1, sizeof(int32_t));
  for (int64_t r = 0; r < rows; r++)
    if (g.row2e[r] >= 0) { phi[g.row2e[r]] = truss_rows[r]; sup[g.row2e[r]] = support_rows[r]; }
  int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.n + 1));
  for (int64_t v = 0; v < g.n; v++) mark[v] = -1;
  /* count, for each edge, triangles whose other edges have phi >= its phi */
  for (int32_t u = 0; u < (int32_t)g.n; u++) {
    for (int64_t j = g.off[u]; j < g.off[u + 1]; j++) mark[g.adj[j]] = g.adje[j];
    for (int64_t j = g.off[u]; j < g.off[u + 1]; j++) {
      int32_t v = g.adj[j];
      if (!before(&g, u, v)) continue;
      int32_t a = g.adje[j];
      for (int64_t q = g.off[v]; q < g.off[v + 1]; q++) {
        int32_t w = g.adj[q];
        if (!before(&g, v, w) || mark[w] < 0) continue;
        int32_t b = mark[w], c = g.adje[q]; /* a=(u,v) b=(u,w) c=(v,w) */
        if (phi[b] >= phi[a] && phi[c] >= phi[a]) in[a]++;
        if (phi[a] >= phi[b] && phi[c] >= phi[b]) in[b]++;
        if (phi[a] >= phi[c] && phi[b] >= phi[c]) in[c]++;
      }
    }
    for (int64_t j = g.off[u]; j < g.off[u + 1]; j++) mark[g.adj[j]] = -1;
  }
  int64_t bad = 0;
  for (int64_t e = 0; e < g.m; e++) {
    int ok = in[e] >= phi[e] - 2 && phi[e] >= 2 && phi[e] <= sup[e] + 2 &&
             ((phi[e] == 2) == (sup[e] == 0));
    if (!ok) bad++;
  }
  free(phi); free(sup); free(in); free(mark);
  g_free(&g);
  return bad;
}

/* Sampled check of a claimed result at any size (Definitions 1 and 2): for
 * each sampled row r (not a self-loop) with edge e = (u, v), its support is
 * |nb(u) cap nb(v)| (merge of the two sorted lists), and e must lie in
 * >= phi(e) - 2 triangles whose other two edges have phi >= phi(e); phi = 2
 * iff the support is 0.  Writes the exact support of each sampled row to
 * sup_sample and returns the number of sampled rows violating any check. */
int64_t oracle_check_sample(int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
                            const int32_t *truss_rows, const int32_t *support_rows,
                            int64_t ns, const int64_t *sample, int32_t *sup_sample) {
  graph g;
  if (g_build(&g, n, rows, src, dst)) { g_free(&g); return -1; }
  int32_t *phi = (int32_t *)malloc(sizeof(int32_t) * (size_t)(g.m + 1));
  for (int64_t r = 0; r < rows; r++)
    if (g.row2e[r] >= 0) phi[g.row2e[r]] = truss_rows[r];
  int64_t bad = 0;
  for (int64_t t = 0; t < ns; t++) {
    const int64_t r = sample[t];
    const int32_t e = g.row2e[r];
    if (e < 0) { sup_sample[t] = -1; bad += truss_rows[r] != -1 || support_rows[r] != -1; continue; }
    const int32_t u = g.eu[e], v = g.ev[e];
    const int32_t pe = truss_rows[r];  /* the sampled row's own claim */
    int64_t i = g.off[u], j = g.off[v];
    int32_t sup = 0, in = 0;
    while (i < g.off[u + 1] && j < g.off[v + 1]) {
      const int32_t a = g.adj[i], b = g.adj[j];
      if (a < b) i++;
      else if (a > b) j++;
      else {
        sup++;
        if (phi[g.adje[i]] >= pe && phi[g.adje[j]] >= pe) in++;
        i++; j++;
      }
    }
    sup_sample[t] = sup;
    const int ok = support_rows[r] == sup && pe >= 2 && pe <= sup + 2 && in >= pe - 2 &&
                   ((pe == 2) == (sup == 0)) && phi[e] == pe;  /* duplicates agree */
    bad += !ok;
  }
  free(phi);
  g_free(&g);
  return bad;
}
