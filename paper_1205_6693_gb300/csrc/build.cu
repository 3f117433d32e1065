// CSR build: from an edge list of rows to the degree-ordered oriented CSR.
//
// The paper assumes adjacency lists already exist (Section 2) and bounds the
// work of Algorithm 2 through the degree order of Theorem 1: orienting every
// edge from its lower-degree to its higher-degree endpoint bounds each vertex's
// out-list by 2*sqrt(m).  Steps:
//   1. canonical key (min, max) per row; self-loops and invalid rows get a
//      sentinel key; radix sort (key, row);
//   2. run heads -> distinct edges in lexicographic order, row -> lex id;
//   3. degrees; rank = position in ascending (degree, id) (stable radix sort
//      by degree over ids in order), vertices relabelled by rank;
//   4. oriented keys (rank tail, rank head), radix sort -> canonical edge id =
//      position; out-degree count + exclusive scan -> offsets;
//   5. row -> canonical edge id.
#include "engine.h"

namespace tr {

namespace {

constexpr int kBlock = 256;

// Graph of row r in a batch (row_off has G+1 entries).
__device__ __forceinline__ int graph_of_row(const int64_t *row_off, int G, int64_t r) {
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (row_off[mid] <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_make_keys(RowsIn in, int b, uint64_t sentinel, uint64_t *keys, int32_t *vals,
                            int32_t *err) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < in.rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t u = in.src[r], v = in.dst[r];
    int64_t lo = 0, hi = in.n;
    if (in.graphs > 1 || in.voff != nullptr) {
      int g = graph_of_row(in.row_off, in.graphs, r);
      lo = in.voff[g];
      hi = in.voff[g + 1];
      u += lo;
      v += lo;
    }
    uint64_t key = sentinel;
    if (u < lo || u >= hi || v < lo || v >= hi) {
      atomicExch(err, TRUSS_EINVAL);
    } else if (u != v) {
      uint64_t a = (uint64_t)(u < v ? u : v), c = (uint64_t)(u < v ? v : u);
      key = (a << b) | c;
    }
    keys[r] = key;
    vals[r] = (int32_t)r;
  }
}

__global__ void k_run_heads(int64_t rows, const uint64_t *sk, uint64_t sentinel, int32_t *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = sk[i];
    flag[i] = (k != sentinel && (i == 0 || sk[i - 1] != k)) ? 1 : 0;
  }
}

// Distinct edges in lexicographic order (U, V) from the sorted row keys;
// runid[i] becomes the 1-based edge id of sorted row i, 0 for a self-loop.
__global__ void k_lex_edges(int64_t rows, const uint64_t *sk, int32_t *runid, uint64_t sentinel,
                            int b, int32_t *U, int32_t *V) {
  const uint64_t mask = (b >= 64) ? ~0ull : ((1ull << b) - 1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = sk[i];
    if (k == sentinel) {
      runid[i] = 0;
      continue;
    }
    int32_t id = runid[i] - 1;
    if (i == 0 || sk[i - 1] != k) {
      U[id] = (int32_t)(k >> b);
      V[id] = (int32_t)(k & mask);
    }
  }
}

// U is sorted (edges in lexicographic order), so each run of equal tails
// adds its length once: minus its first index at its first edge, its end at
// its last (int32 wrap-around cancels).  Heads V are added once per group of
// lanes of a warp that hold the same vertex.
__global__ void k_degree(int64_t m, const int32_t *U, const int32_t *V, int32_t *deg) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x; b < m; b += stride) {
    const int64_t e = b + threadIdx.x;
    const bool ok = e < m;
    if (ok) {
      const int u = U[e];
      if (e == 0 || U[e - 1] != u) atomicAdd(&deg[u], -(int)e);
      if (e + 1 == m || U[e + 1] != u) atomicAdd(&deg[u], (int)(e + 1));
    }
    const int v = ok ? V[e] : -1;
    const unsigned peers = __match_any_sync(TR_FULL, v);
    if (ok && lane_id() == __ffs(peers) - 1) atomicAdd(&deg[v], __popc(peers));
  }
}

__global__ void k_iota(int64_t n, int32_t *x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = (int32_t)i;
}

__global__ void k_newid(int64_t n, const int32_t *order, int32_t *newid) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    newid[order[i]] = (int32_t)i;
}

__global__ void k_orient_keys(int64_t m, const int32_t *U, const int32_t *V, const int32_t *newid,
                              int b, uint64_t *keys, int32_t *vals) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t x = (uint64_t)newid[U[e]], y = (uint64_t)newid[V[e]];
    keys[e] = x < y ? ((x << b) | y) : ((y << b) | x);
    vals[e] = (int32_t)e;
  }
}

// The oriented edges are sorted by tail, so each run of equal tails adds
// its length to outdeg once: minus its first index at its first edge, its
// end at its last.
__global__ void k_oriented(int64_t m, const uint64_t *ok, const int32_t *olex, int b,
                           int32_t *adjp, int32_t *esrc, int32_t *lex2e, int64_t *outdeg) {
  const uint64_t mask = (1ull << b) - 1;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m;
       p += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = ok[p];
    int32_t x = (int32_t)(k >> b), y = (int32_t)(k & mask);
    adjp[p] = y;
    esrc[p] = x;
    lex2e[olex[p]] = (int32_t)p;
    if (p == 0 || (int32_t)(ok[p - 1] >> b) != x)
      atomicAdd((unsigned long long *)&outdeg[x], (unsigned long long)(-p));
    if (p + 1 == m || (int32_t)(ok[p + 1] >> b) != x)
      atomicAdd((unsigned long long *)&outdeg[x], (unsigned long long)(p + 1));
  }
}

// Row srow[i] (sorted row i) -> its canonical edge: the lexicographic id is
// runid[i] - 1 (0: a self-loop), read in order, so lex2e is read in order
// and only the write to row2e lands at random.
__global__ void k_row2e(int64_t rows, const int32_t *srow, const int32_t *runid,
                        const int32_t *lex2e, int32_t *row2e) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t l = runid[i];
    row2e[srow[i]] = l > 0 ? lex2e[l - 1] : -1;
  }
}

}  // namespace

int build_csr(Arena &A, const RowsIn &in, Csr *out, int32_t *d_err, cudaStream_t s) {
  const int64_t rows = in.rows, n = in.n;
  const int maxg = 152 * 16;
  out->n = n;
  out->rows = rows;
  const int b = bits_for(n > 1 ? (uint64_t)(n - 1) : 1);
  const uint64_t sentinel = (2 * b >= 64) ? ~0ull : ((1ull << (2 * b)) - 1);

  int32_t *row2e = A.get<int32_t>(rows);
  int64_t *offp = A.get<int64_t>(n + 1);
  if (!row2e || !offp) return TRUSS_ENOMEM;
  out->row2e = row2e;
  out->offp = offp;

  if (rows == 0) {
    // no edges: empty out-lists, and every vertex keeps its id as its rank
    int32_t *order = A.get<int32_t>(n);
    if (!order) return TRUSS_ENOMEM;
    TR_CUDA(cudaMemsetAsync(offp, 0, sizeof(int64_t) * (n + 1), s));
    if (n > 0) {
      k_iota<<<grid_for(n, kBlock, maxg), kBlock, 0, s>>>(n, order);
      TR_LAUNCHED();
    }
    out->m = 0;
    out->order = order;
    out->adjp = A.get<int32_t>(1);
    out->esrc = A.get<int32_t>(1);
    return TRUSS_OK;
  }

  // 1. keys + sort
  uint64_t *keys = A.get<uint64_t>(rows), *skeys = A.get<uint64_t>(rows);
  int32_t *vals = A.get<int32_t>(rows), *srow = A.get<int32_t>(rows);
  int32_t *flag = A.get<int32_t>(rows), *runid = A.get<int32_t>(rows);
  if (!keys || !skeys || !vals || !srow || !flag || !runid) return TRUSS_ENOMEM;
  k_make_keys<<<grid_for(rows, kBlock, maxg), kBlock, 0, s>>>(in, b, sentinel, keys, vals, d_err);
  TR_LAUNCHED();
  size_t tb = 0;
  TR_TRY(sort_pairs_u64(nullptr, &tb, keys, skeys, vals, srow, rows, 0, 2 * b, s));
  void *tmp = A.alloc(tb);
  if (!tmp) return TRUSS_ENOMEM;
  TR_TRY(sort_pairs_u64(tmp, &tb, keys, skeys, vals, srow, rows, 0, 2 * b, s));

  // 2. distinct edges
  k_run_heads<<<grid_for(rows, kBlock, maxg), kBlock, 0, s>>>(rows, skeys, sentinel, flag);
  TR_LAUNCHED();
  tb = 0;
  TR_TRY(inclusive_sum_i32(nullptr, &tb, flag, runid, rows, s));
  tmp = A.alloc(tb);
  if (!tmp) return TRUSS_ENOMEM;
  TR_TRY(inclusive_sum_i32(tmp, &tb, flag, runid, rows, s));
  int32_t h_m = 0, h_err = 0;
  TR_CUDA(cudaMemcpyAsync(&h_m, runid + rows - 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  if (h_err != 0) return TRUSS_EINVAL;
  const int64_t m = h_m;
  out->m = m;
  int32_t *U = A.get<int32_t>(m), *V = A.get<int32_t>(m);
  if (!U || !V) return TRUSS_ENOMEM;
  k_lex_edges<<<grid_for(rows, kBlock, maxg), kBlock, 0, s>>>(rows, skeys, runid, sentinel, b, U,
                                                               V);
  TR_LAUNCHED();

  // 3. degrees and rank
  int32_t *deg = A.get<int32_t>(n), *sdeg = A.get<int32_t>(n);
  int32_t *ids = A.get<int32_t>(n), *order = A.get<int32_t>(n), *newid = A.get<int32_t>(n);
  if (!deg || !sdeg || !ids || !order || !newid) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * n, s));
  if (m > 0) {
    k_degree<<<grid_for(m, kBlock, maxg), kBlock, 0, s>>>(m, U, V, deg);
    TR_LAUNCHED();
  }
  k_iota<<<grid_for(n, kBlock, maxg), kBlock, 0, s>>>(n, ids);
  TR_LAUNCHED();
  const int db = bits_for((uint64_t)(m > 0 ? m : 1));
  tb = 0;
  TR_TRY(sort_pairs_u32(nullptr, &tb, (const uint32_t *)deg, (uint32_t *)sdeg, ids, order, n, 0,
                        db, s));
  tmp = A.alloc(tb);
  if (!tmp) return TRUSS_ENOMEM;
  TR_TRY(sort_pairs_u32(tmp, &tb, (const uint32_t *)deg, (uint32_t *)sdeg, ids, order, n, 0, db,
                        s));
  out->order = order;
  k_newid<<<grid_for(n, kBlock, maxg), kBlock, 0, s>>>(n, order, newid);
  TR_LAUNCHED();

  // 4. orientation
  int32_t *adjp = A.get<int32_t>(m), *esrc = A.get<int32_t>(m), *lex2e = A.get<int32_t>(m);
  int64_t *outdeg = A.get<int64_t>(n + 1);
  if (!adjp || !esrc || !lex2e || !outdeg) return TRUSS_ENOMEM;
  out->adjp = adjp;
  out->esrc = esrc;
  TR_CUDA(cudaMemsetAsync(outdeg, 0, sizeof(int64_t) * (n + 1), s));
  if (m > 0) {
    // reuse the row-sized key/value buffers (m <= rows); srow and runid
    // stay for the row -> edge map, flag (dead) takes the sorted values
    int32_t *olex = flag;
    k_orient_keys<<<grid_for(m, kBlock, maxg), kBlock, 0, s>>>(m, U, V, newid, b, keys, vals);
    TR_LAUNCHED();
    tb = 0;
    TR_TRY(sort_pairs_u64(nullptr, &tb, keys, skeys, vals, olex, m, 0, 2 * b, s));
    tmp = A.alloc(tb);
    if (!tmp) return TRUSS_ENOMEM;
    TR_TRY(sort_pairs_u64(tmp, &tb, keys, skeys, vals, olex, m, 0, 2 * b, s));
    k_oriented<<<grid_for(m, kBlock, maxg), kBlock, 0, s>>>(m, skeys, olex, b, adjp, esrc, lex2e,
                                                             outdeg);
    TR_LAUNCHED();
  }
  tb = 0;
  TR_TRY(exclusive_sum_i64(nullptr, &tb, outdeg, offp, n + 1, s));
  tmp = A.alloc(tb);
  if (!tmp) return TRUSS_ENOMEM;
  TR_TRY(exclusive_sum_i64(tmp, &tb, outdeg, offp, n + 1, s));

  // 5. rows -> canonical edge ids
  k_row2e<<<grid_for(rows, kBlock, maxg), kBlock, 0, s>>>(rows, srow, runid, lex2e, row2e);
  TR_LAUNCHED();
  return TRUSS_OK;
}

}  // namespace tr
