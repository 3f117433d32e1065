// Upper bound psi and candidate subgraphs for the top-t truss classes
// (Section 6: Procedure 6, Algorithm 7, Lemma 2).
//
// psi(e) = min{sup(e), x_u, x_v} + 2, where x_w is the largest x such that
// w has x incident edges other than e with support >= x (Procedure 6, with
// the whole graph as the neighbourhood subgraph: every edge is internal).
// Per vertex w this is the h-index of the supports of its incident edges
// with one of them left out.  With h_w the h-index of all of them and c_w the
// number of incident supports >= h_w, leaving out an edge of support s gives
// h_w - 1 when s >= h_w and c_w == h_w (only h_w - 1 supports >= h_w remain,
// and at least h_w - 1 are >= h_w - 1), and h_w otherwise.  So one h-index
// per vertex gives x_u and x_v of every edge.
//
// Lemma 2 gives phi(e) <= psi(e): the k-truss T_k of G lies inside
// G_k = {e : psi(e) >= k}, and is therefore also the k-truss of any
// subgraph between G_k and G.  Decomposing the subgraph {e : psi(e) >= k_lo}
// thus yields every truss number >= k_lo exactly (the ones below k_lo are
// not meaningful there).
#include <climits>

#include "engine.h"

namespace tr {

namespace {

constexpr int kBlk = 128;

__global__ void k_in_count(int64_t m, const int32_t *adjp, unsigned long long *indeg) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&indeg[adjp[e]], 1ull);
}

// inedge[inoff[v] ..) = the oriented edges (u, v) with head v, in any order.
__global__ void k_in_fill(int64_t m, const int32_t *adjp, const int64_t *inoff,
                          unsigned long long *cur, int32_t *inedge) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int v = adjp[e];
    const unsigned long long p = atomicAdd(&cur[v], 1ull);
    inedge[inoff[v] + (int64_t)p] = (int32_t)e;
  }
}

// Block sum of one value per thread.
__device__ __forceinline__ int block_sum(int x, int *red) {
  for (int o = 16; o >= 1; o >>= 1) x += __shfl_down_sync(TR_FULL, x, o);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if (lane_id() == 0) red[w] = x;
  __syncthreads();
  int t = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += red[i];
  return t;
}

// Supports of the edges incident to w that are >= x: out-edges are the
// contiguous range offp[w] .. offp[w+1], in-edges come through inedge.
__device__ __forceinline__ int count_ge(const int32_t *sup, int64_t ob, int dout,
                                        const int32_t *inedge, int64_t ib, int din, int x,
                                        int *red) {
  int c = 0;
  for (int i = threadIdx.x; i < dout; i += blockDim.x) c += __ldg(&sup[ob + i]) >= x;
  for (int i = threadIdx.x; i < din; i += blockDim.x)
    c += __ldg(&sup[__ldg(&inedge[ib + i])]) >= x;
  return block_sum(c, red);
}

// h_w (h-index of the incident supports) and c_w (how many are >= h_w):
// bisection on x over [0, deg(w)], since #{supports >= x} >= x holds exactly
// for x <= h_w.  Vertices of degree <= kRegVals * 32 take one warp, with the
// supports held in registers; larger ones take a whole block and re-read the
// supports at every step.
constexpr int kRegVals = 8;

__global__ void __launch_bounds__(256) k_hindex_warp(int64_t n, const int64_t *offp,
                                                     const int64_t *inoff, const int32_t *inedge,
                                                     const int32_t *sup, int32_t *h, int32_t *c,
                                                     int32_t *big, unsigned long long *nbig) {
  const int lane = lane_id();
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = gw; w < n; w += nw) {
    const int64_t ob = offp[w], ib = inoff[w];
    const int dout = (int)(offp[w + 1] - ob), din = (int)(inoff[w + 1] - ib);
    const int d = dout + din;
    if (d > kRegVals * 32) {
      if (lane == 0) big[atomicAdd(nbig, 1ull)] = (int32_t)w;
      continue;
    }
    int val[kRegVals];
#pragma unroll
    for (int k = 0; k < kRegVals; k++) {
      const int i = k * 32 + lane;
      val[k] = i < dout ? __ldg(&sup[ob + i])
               : i < d  ? __ldg(&sup[__ldg(&inedge[ib + i - dout])])
                        : -1;
    }
    int lo = 0, hi = d + 1, clo = d;
    while (hi - lo > 1) {
      const int mid = lo + ((hi - lo) >> 1);
      int cm = 0;
#pragma unroll
      for (int k = 0; k < kRegVals; k++) cm += val[k] >= mid;
      cm = __reduce_add_sync(TR_FULL, cm);
      if (cm >= mid) {
        lo = mid;
        clo = cm;
      } else {
        hi = mid;
      }
    }
    if (lane == 0) {
      h[w] = lo;
      c[w] = clo;
    }
  }
}

// The vertices k_hindex_warp left out (degree > kRegVals * 32), one block each.
__global__ void __launch_bounds__(kBlk) k_hindex_block(const int32_t *big,
                                                       const unsigned long long *nbig,
                                                       const int64_t *offp, const int64_t *inoff,
                                                       const int32_t *inedge, const int32_t *sup,
                                                       int32_t *h, int32_t *c) {
  __shared__ int red[kBlk / 32];
  const int64_t nb = (int64_t)*nbig;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const int64_t w = big[b];
    const int64_t ob = offp[w], ib = inoff[w];
    const int dout = (int)(offp[w + 1] - ob), din = (int)(inoff[w + 1] - ib);
    const int d = dout + din;
    int lo = 0, hi = d + 1, clo = d;
    while (hi - lo > 1) {
      const int mid = lo + ((hi - lo) >> 1);
      const int cm = count_ge(sup, ob, dout, inedge, ib, din, mid, red);
      if (cm >= mid) {
        lo = mid;
        clo = cm;
      } else {
        hi = mid;
      }
    }
    if (threadIdx.x == 0) {
      h[w] = lo;
      c[w] = clo;
    }
  }
}

__device__ __forceinline__ int x_without(int hw, int cw, int s) {
  return hw - ((s >= hw && cw == hw) ? 1 : 0);
}

__global__ void k_psi(int64_t m, const int32_t *esrc, const int32_t *adjp, const int32_t *sup,
                      const int32_t *h, const int32_t *c, int32_t *psi) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int u = esrc[e], v = adjp[e], s = sup[e];
    const int xu = x_without(h[u], c[u], s), xv = x_without(h[v], c[v], s);
    psi[e] = min(s, min(xu, xv)) + 2;
  }
}

__global__ void k_max_i32(int64_t m, const int32_t *x, int *out) {
  int mx = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, x[e]);
  mx = __reduce_max_sync(TR_FULL, mx);
  if (lane_id() == 0) atomicMax(out, mx);
}

// Histogram of x[0 .. m): per-block counts in shared memory for the first
// kHistBins values (most edges share a few small psi values, and global
// atomics on one address would serialise), global atomics above.
constexpr int kHistBins = 4096;

__global__ void k_hist(int64_t m, const int32_t *x, unsigned long long *hist, int nbins) {
  __shared__ unsigned s_hist[kHistBins];
  const int lim = nbins < kHistBins ? nbins : kHistBins;
  for (int i = threadIdx.x; i < lim; i += blockDim.x) s_hist[i] = 0;
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int v = x[e];
    if (v < lim) atomicAdd(&s_hist[v], 1u);
    else atomicAdd(&hist[v], 1ull);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < lim; i += blockDim.x)
    if (s_hist[i]) atomicAdd(&hist[i], (unsigned long long)s_hist[i]);
}

__global__ void k_select(int64_t m, const int32_t *esrc, const int32_t *adjp, const int32_t *psi,
                         int k_lo, unsigned long long *cnt, int32_t *cs, int32_t *cd,
                         int32_t *ce) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x; b < m; b += stride) {
    const int64_t e = b + threadIdx.x;
    const bool take = e < m && psi[e] >= k_lo;
    const long long p = warp_append64(take, cnt);
    if (take) {
      cs[p] = esrc[e];
      cd[p] = adjp[e];
      ce[p] = (int32_t)e;
    }
  }
}

__global__ void k_top(int64_t mc, const int32_t *ce, const int32_t *phi_rows, int thr,
                      int32_t *top) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < mc;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int v = phi_rows[r];
    top[ce[r]] = v >= thr ? v : 0;
  }
}

}  // namespace

int compute_psi(Arena &A, const Csr &g, const int32_t *sup, int32_t *psi, cudaStream_t s) {
  const int64_t m = g.m, n = g.n;
  if (m == 0) return TRUSS_OK;
  unsigned long long *cnt = A.get<unsigned long long>(n + 1);
  int64_t *inoff = A.get<int64_t>(n + 1);
  int32_t *inedge = A.get<int32_t>(m), *h = A.get<int32_t>(n), *c = A.get<int32_t>(n);
  if (!cnt || !inoff || !inedge || !h || !c) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (n + 1), s));
  k_in_count<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, g.adjp, cnt);
  TR_LAUNCHED();
  size_t tb = 0;
  TR_TRY(exclusive_sum_i64(nullptr, &tb, (const int64_t *)cnt, inoff, n + 1, s));
  void *tmp = A.alloc(tb);
  if (!tmp) return TRUSS_ENOMEM;
  TR_TRY(exclusive_sum_i64(tmp, &tb, (const int64_t *)cnt, inoff, n + 1, s));
  TR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (n + 1), s));
  k_in_fill<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, g.adjp, inoff, cnt, inedge);
  TR_LAUNCHED();
  if (n > 0) {
    int32_t *big = A.get<int32_t>(n);
    unsigned long long *nbig = A.get<unsigned long long>(1);
    if (!big || !nbig) return TRUSS_ENOMEM;
    TR_CUDA(cudaMemsetAsync(nbig, 0, sizeof(unsigned long long), s));
    k_hindex_warp<<<grid_for(n * 32, 256, 152 * 16), 256, 0, s>>>(n, g.offp, inoff, inedge, sup,
                                                                  h, c, big, nbig);
    TR_LAUNCHED();
    k_hindex_block<<<152 * 8, kBlk, 0, s>>>(big, nbig, g.offp, inoff, inedge, sup, h, c);
    TR_LAUNCHED();
  }
  k_psi<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, g.esrc, g.adjp, sup, h, c, psi);
  TR_LAUNCHED();
  return TRUSS_OK;
}

int psi_counts(Arena &A, int64_t m, const int32_t *psi, std::vector<int64_t> *cnt_ge,
               cudaStream_t s) {
  cnt_ge->assign(1, m);
  if (m == 0) return TRUSS_OK;
  int *mx = A.get<int>(1);
  if (!mx) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(mx, 0, sizeof(int), s));
  k_max_i32<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, psi, mx);
  TR_LAUNCHED();
  int hmx = 0;
  TR_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(int), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  unsigned long long *hist = A.get<unsigned long long>((int64_t)hmx + 1);
  if (!hist) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * ((size_t)hmx + 1), s));
  k_hist<<<grid_for(m, 256, 152 * 4), 256, 0, s>>>(m, psi, hist, hmx + 1);
  TR_LAUNCHED();
  std::vector<unsigned long long> hh((size_t)hmx + 1);
  TR_CUDA(cudaMemcpyAsync(hh.data(), hist, sizeof(unsigned long long) * hh.size(),
                          cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  cnt_ge->assign((size_t)hmx + 2, 0);
  for (int k = hmx; k >= 0; k--) (*cnt_ge)[k] = (*cnt_ge)[k + 1] + (int64_t)hh[k];
  cnt_ge->pop_back();
  return TRUSS_OK;
}

int select_candidates(Arena &A, const Csr &g, const int32_t *psi, int32_t k_lo, int32_t *cs,
                      int32_t *cd, int32_t *ce, int64_t *mc, cudaStream_t s) {
  *mc = 0;
  if (g.m == 0) return TRUSS_OK;
  unsigned long long *cnt = A.get<unsigned long long>(1);
  if (!cnt) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  k_select<<<grid_for(g.m, 256, 152 * 16), 256, 0, s>>>(g.m, g.esrc, g.adjp, psi, k_lo, cnt, cs,
                                                         cd, ce);
  TR_LAUNCHED();
  unsigned long long h = 0;
  TR_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  *mc = (int64_t)h;
  return TRUSS_OK;
}

int top_classes(int64_t m, int64_t mc, const int32_t *ce, const int32_t *phi_rows, int32_t thr,
                int32_t *top, cudaStream_t s) {
  if (m == 0) return TRUSS_OK;
  TR_CUDA(cudaMemsetAsync(top, 0, sizeof(int32_t) * m, s));
  if (mc > 0) {
    k_top<<<grid_for(mc, 256, 152 * 16), 256, 0, s>>>(mc, ce, phi_rows, thr, top);
    TR_LAUNCHED();
  }
  return TRUSS_OK;
}

}  // namespace tr
