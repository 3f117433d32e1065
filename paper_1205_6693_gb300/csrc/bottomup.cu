// Kernels of the bottom-up decomposition under a working-set budget
// (Section 5: Algorithm 3 LowerBounding, Algorithm 4 and Procedure 5), used
// when the decomposition's working set of a whole graph would not fit in
// device memory.  The host side (api.cu: run_bottom_up) chooses the
// neighbourhood subgraphs and runs the in-memory pipeline on each; these
// kernels select their edges and fold the results back.
//
// Edge state: 0 = still in the graph G of Algorithm 3, 1 = in G_new with a
// lower bound (Algorithm 3 step 10), 2 = truss number known.
#include <climits>

#include "engine.h"

namespace tr {

namespace {

__global__ void k_bu_list_state(int64_t m, const uint8_t *state, int want,
                                unsigned long long *cnt, int32_t *out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x; b < m; b += stride) {
    const int64_t e = b + threadIdx.x;
    const bool take = e < m && state[e] == want;
    const long long p = warp_append64(take, cnt);
    if (take) out[p] = (int32_t)e;
  }
}

__global__ void k_bu_degrees(int64_t nl, const int32_t *list, const int32_t *eu,
                             const int32_t *ev, int32_t *deg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int e = list[i];
    atomicAdd(&deg[eu[e]], 1);
    atomicAdd(&deg[ev[e]], 1);
  }
}

// Edges of `list` with an endpoint in [va, vb): the neighbourhood subgraph
// of that vertex range (Definition 4).
__global__ void k_bu_select_range(int64_t nl, const int32_t *list, const int32_t *eu,
                                  const int32_t *ev, int32_t va, int32_t vb,
                                  unsigned long long *cnt, int32_t *hs, int32_t *hd,
                                  int32_t *hid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x; b < nl; b += stride) {
    const int64_t i = b + threadIdx.x;
    int e = -1, u = 0, v = 0;
    if (i < nl) {
      e = list[i];
      u = eu[e];
      v = ev[e];
    }
    const bool take = e >= 0 && ((u >= va && u < vb) || (v >= va && v < vb));
    const long long p = warp_append64(take, cnt);
    if (take) {
      hs[p] = u;
      hd[p] = v;
      hid[p] = e;
    }
  }
}

// Algorithm 3 steps 7-10 for one neighbourhood subgraph H = NS([va, vb)):
// every edge of H raises its lower bound to its truss number in H (Lemma 1),
// and the internal edges (both ends in the range) leave G: to Phi_2 if
// their lower bound is still 2, to G_new otherwise.
// Reading of step 8: its support test is made on the bound, not on the
// support in H.  G shrinks from pass to pass, so an edge can have support 0
// in H while its triangles' other edges already left G; but when the first
// edge of a triangle left G, the H of that step held the whole triangle and
// raised all three bounds to at least 3.  A bound of 2 therefore means no
// triangle at all.
__global__ void k_bu_alg3_update(int64_t mh, const int32_t *hid, const int32_t *hs,
                                 const int32_t *hd, int32_t va, int32_t vb,
                                 const int32_t *truss_h, int32_t *lower, int32_t *phi,
                                 uint8_t *state) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < mh;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int e = hid[r];
    const int low = max(atomicMax(&lower[e], truss_h[r]), truss_h[r]);
    const bool internal = hs[r] >= va && hs[r] < vb && hd[r] >= va && hd[r] < vb;
    if (internal) {
      if (low <= 2) {
        phi[e] = 2;
        state[e] = 2;
      } else {
        state[e] = 1;
      }
    }
  }
}

__global__ void k_bu_min_lower(int64_t nl, const int32_t *list, const int32_t *lower,
                               int *out) {
  int mn = INT_MAX;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl;
       i += (int64_t)gridDim.x * blockDim.x)
    mn = min(mn, lower[list[i]]);
  mn = __reduce_min_sync(TR_FULL, mn);
  if (lane_id() == 0) atomicMin(out, mn);
}

// U_k of Algorithm 4 step 3: endpoints of G_new edges with lower bound <= k.
__global__ void k_bu_mark(int64_t nl, const int32_t *list, const int32_t *eu, const int32_t *ev,
                          const int32_t *lower, int k, uint8_t *inU) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int e = list[i];
    if (lower[e] <= k) {
      inU[eu[e]] = 1;
      inU[ev[e]] = 1;
    }
  }
}

// H = NS(U_k) within G_new (Algorithm 4 steps 4-5); its external edges
// (one end outside U_k) are pinned for Procedure 5.
__global__ void k_bu_select_marked(int64_t nl, const int32_t *list, const int32_t *eu,
                                   const int32_t *ev, const uint8_t *inU,
                                   unsigned long long *cnt, int32_t *hs, int32_t *hd,
                                   int32_t *hid, uint8_t *pinned) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x; b < nl; b += stride) {
    const int64_t i = b + threadIdx.x;
    int e = -1, u = 0, v = 0;
    bool iu = false, iv = false;
    if (i < nl) {
      e = list[i];
      u = eu[e];
      v = ev[e];
      iu = inU[u] != 0;
      iv = inU[v] != 0;
    }
    const bool take = e >= 0 && (iu || iv);
    const long long p = warp_append64(take, cnt);
    if (take) {
      hs[p] = u;
      hd[p] = v;
      hid[p] = e;
      pinned[p] = (iu && iv) ? 0 : 1;
    }
  }
}

// Procedure 5's output: internal edges removed at threshold k are Phi_k.
__global__ void k_bu_assign(int64_t mh, const int32_t *hid, const uint8_t *pinned,
                            const int32_t *truss_h, int k, int32_t *phi, uint8_t *state) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < mh;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (!pinned[r] && truss_h[r] > 0) {
      const int e = hid[r];
      phi[e] = k;
      state[e] = 2;
    }
  }
}

__global__ void k_bu_max(int64_t m, const int32_t *x, int *out) {
  int mx = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, x[e]);
  mx = __reduce_max_sync(TR_FULL, mx);
  if (lane_id() == 0) atomicMax(out, mx);
}

__global__ void k_pin_edges(int64_t rows, const int32_t *row2e, const uint8_t *pinned_rows,
                            uint8_t *pinned_e) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int e = row2e[r];
    if (e >= 0 && pinned_rows[r]) pinned_e[e] = 1;
  }
}

}  // namespace

int bu_list_state(Arena &A, int64_t m, const uint8_t *state, int want, int32_t *out,
                  int64_t *count, cudaStream_t s) {
  *count = 0;
  if (m == 0) return TRUSS_OK;
  unsigned long long *cnt = A.get<unsigned long long>(1);
  if (!cnt) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  k_bu_list_state<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, state, want, cnt, out);
  TR_LAUNCHED();
  unsigned long long h = 0;
  TR_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  *count = (int64_t)h;
  return TRUSS_OK;
}

int bu_degrees(int64_t n, int64_t nl, const int32_t *list, const int32_t *eu, const int32_t *ev,
               int32_t *deg, cudaStream_t s) {
  TR_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (n > 0 ? n : 1), s));
  if (nl > 0) {
    k_bu_degrees<<<grid_for(nl, 256, 152 * 16), 256, 0, s>>>(nl, list, eu, ev, deg);
    TR_LAUNCHED();
  }
  return TRUSS_OK;
}

int bu_select_range(Arena &A, int64_t nl, const int32_t *list, const int32_t *eu,
                    const int32_t *ev, int32_t va, int32_t vb, int32_t *hs, int32_t *hd,
                    int32_t *hid, int64_t *mh, cudaStream_t s) {
  *mh = 0;
  if (nl == 0) return TRUSS_OK;
  unsigned long long *cnt = A.get<unsigned long long>(1);
  if (!cnt) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  k_bu_select_range<<<grid_for(nl, 256, 152 * 16), 256, 0, s>>>(nl, list, eu, ev, va, vb, cnt,
                                                                hs, hd, hid);
  TR_LAUNCHED();
  unsigned long long h = 0;
  TR_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  *mh = (int64_t)h;
  return TRUSS_OK;
}

int bu_alg3_update(int64_t mh, const int32_t *hid, const int32_t *hs, const int32_t *hd,
                   int32_t va, int32_t vb, const int32_t *truss_h, int32_t *lower, int32_t *phi,
                   uint8_t *state, cudaStream_t s) {
  if (mh == 0) return TRUSS_OK;
  k_bu_alg3_update<<<grid_for(mh, 256, 152 * 16), 256, 0, s>>>(mh, hid, hs, hd, va, vb, truss_h,
                                                               lower, phi, state);
  TR_LAUNCHED();
  return TRUSS_OK;
}

int bu_min_lower(Arena &A, int64_t nl, const int32_t *list, const int32_t *lower, int32_t *mn,
                 cudaStream_t s) {
  *mn = INT_MAX;
  if (nl == 0) return TRUSS_OK;
  int *d = A.get<int>(1);
  if (!d) return TRUSS_ENOMEM;
  const int init = INT_MAX;
  TR_CUDA(cudaMemcpyAsync(d, &init, sizeof(int), cudaMemcpyHostToDevice, s));
  k_bu_min_lower<<<grid_for(nl, 256, 152 * 16), 256, 0, s>>>(nl, list, lower, d);
  TR_LAUNCHED();
  TR_CUDA(cudaMemcpyAsync(mn, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  return TRUSS_OK;
}

int bu_select_candidates(Arena &A, int64_t n, int64_t nl, const int32_t *list, const int32_t *eu,
                         const int32_t *ev, const int32_t *lower, int32_t k, uint8_t *inU,
                         int32_t *hs, int32_t *hd, int32_t *hid, uint8_t *pinned, int64_t *mh,
                         cudaStream_t s) {
  *mh = 0;
  if (nl == 0) return TRUSS_OK;
  unsigned long long *cnt = A.get<unsigned long long>(1);
  if (!cnt) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(inU, 0, (size_t)(n > 0 ? n : 1), s));
  TR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
  k_bu_mark<<<grid_for(nl, 256, 152 * 16), 256, 0, s>>>(nl, list, eu, ev, lower, k, inU);
  TR_LAUNCHED();
  k_bu_select_marked<<<grid_for(nl, 256, 152 * 16), 256, 0, s>>>(nl, list, eu, ev, inU, cnt, hs,
                                                                 hd, hid, pinned);
  TR_LAUNCHED();
  unsigned long long h = 0;
  TR_CUDA(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  *mh = (int64_t)h;
  return TRUSS_OK;
}

int bu_assign(int64_t mh, const int32_t *hid, const uint8_t *pinned, const int32_t *truss_h,
              int32_t k, int32_t *phi, uint8_t *state, cudaStream_t s) {
  if (mh == 0) return TRUSS_OK;
  k_bu_assign<<<grid_for(mh, 256, 152 * 16), 256, 0, s>>>(mh, hid, pinned, truss_h, k, phi,
                                                          state);
  TR_LAUNCHED();
  return TRUSS_OK;
}

int bu_max(Arena &A, int64_t m, const int32_t *x, int32_t *mx, cudaStream_t s) {
  *mx = 0;
  if (m == 0) return TRUSS_OK;
  int *d = A.get<int>(1);
  if (!d) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(d, 0, sizeof(int), s));
  k_bu_max<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, x, d);
  TR_LAUNCHED();
  TR_CUDA(cudaMemcpyAsync(mx, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  return TRUSS_OK;
}

int pin_edges(int64_t rows, const int32_t *row2e, const uint8_t *pinned_rows, uint8_t *pinned_e,
              int64_t m, cudaStream_t s) {
  TR_CUDA(cudaMemsetAsync(pinned_e, 0, (size_t)(m > 0 ? m : 1), s));
  if (rows > 0) {
    k_pin_edges<<<grid_for(rows, 256, 152 * 16), 256, 0, s>>>(rows, row2e, pinned_rows, pinned_e);
    TR_LAUNCHED();
  }
  return TRUSS_OK;
}

}  // namespace tr
