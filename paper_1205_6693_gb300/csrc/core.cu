// Vertex core numbers on the truss library's CSR.  The paper places the
// k-truss inside the (k-1)-core (Section 1) and compares the k_max-truss with
// the c_max-core (Section 7, Table 6); its edge bins reuse the core
// decomposition's bin-sorted degree array (Section 3.2).
//
// core(v) is the largest k such that v lies in the k-core, the largest
// subgraph whose vertices all have degree >= k in it.  Like the edge peel,
// this runs level-synchronously in one persistent cooperative launch:
//
//  scan (level k):  F = {alive v : deg(v) <= k}; the minimum degree of the
//        other alive vertices lets an empty level jump to k = that minimum.
//        The alive list is rewritten without removed vertices only when at
//        most half of it is still alive.
//  sub-round:  every v in F gets core k and is removed; each neighbour w
//        still alive loses one degree, and a w whose degree crosses from
//        k+1 to k joins the next frontier (it now has degree <= k, so it is
//        not in the k+1-core).  Vertices removed together need no exchange:
//        a neighbour in the same frontier is simply skipped.
//
// Vertex state is stamp[v]: 0 = alive, s = in the frontier of sub-round s,
// 0 < stamp < s = removed earlier; a vertex pushed during sub-round s is
// stamped s+1 and still counts as alive during s.  Neighbours come from a
// symmetric adjacency built from the oriented CSR.  A frontier vertex is
// split into work items of kItem neighbours, as in the edge peel, so a
// warp's share of a sub-round is bounded whatever the degrees.
#include <climits>

#include "engine.h"

namespace tr {

namespace {

constexpr int kBlock = 512;
constexpr int kWarps = kBlock / 32;
constexpr int kItem = 16;  // neighbours per work item (8 lanes x 2)
constexpr int kWQ = 64;    // work items staged per warp
constexpr int kWA = 128;   // alive-list entries staged per warp

struct CoreCtl {
  unsigned long long bar;
  int err;
  int pad0;
  unsigned long long qf[3];  // frontier items appended in phase p (slot p % 3)
  unsigned long long qa[3];  // alive-list entries appended in phase p
  int minres[3];             // per scan (slot = scan index % 3)
  int live[3];
  int levels, subrounds, kmax, pad1;
};

struct CoreArgs {
  int64_t n;
  const int64_t *soff;  // [n+1] symmetric adjacency offsets
  const int32_t *sadj;  // [2m]
  int32_t *deg;         // current degrees (start: full degrees)
  int32_t *stamp;
  int32_t *core;
  int32_t *alive0, *alive1;
  int4 *Q0, *Q1;  // work items (v, cnt | first << 8, offset lo, hi)
  int64_t item_cap;
  CoreCtl *ctl;
  long long wait_ns;
};

__device__ __forceinline__ int items_of(int len) { return len > 0 ? (len + kItem - 1) / kItem : 1; }

struct WarpBuf {
  int4 *items;
  int ni;
  int32_t *alive;
  int na;
};

__device__ __forceinline__ void flush_items(const CoreArgs &a, WarpBuf &wb, int4 *Q,
                                            unsigned long long *qctr) {
  if (wb.ni == 0) return;
  const int lane = lane_id();
  unsigned long long b = 0;
  if (lane == 0) b = atomicAdd(qctr, (unsigned long long)wb.ni);
  const long long b0 = (long long)__shfl_sync(TR_FULL, b, 0);
  for (int t = lane; t < wb.ni; t += 32)
    if (b0 + t < a.item_cap) Q[b0 + t] = wb.items[t];
  __syncwarp();
  wb.ni = 0;
}

__device__ __forceinline__ void flush_alive(const CoreArgs &a, WarpBuf &wb, int32_t *A2,
                                            unsigned long long *actr) {
  if (wb.na == 0) return;
  const int lane = lane_id();
  unsigned long long b = 0;
  if (lane == 0) b = atomicAdd(actr, (unsigned long long)wb.na);
  const long long b0 = (long long)__shfl_sync(TR_FULL, b, 0);
  for (int t = lane; t < wb.na; t += 32)
    if (b0 + t < a.n) A2[b0 + t] = wb.alive[t];
  __syncwarp();
  wb.na = 0;
}

__device__ __forceinline__ void push_alive(const CoreArgs &a, bool keep, int v, WarpBuf &wb,
                                           int32_t *A2, unsigned long long *actr) {
  const unsigned mask = __ballot_sync(TR_FULL, keep);
  if (mask == 0) return;
  const int tot = __popc(mask);
  if (wb.na + tot > kWA) flush_alive(a, wb, A2, actr);
  if (keep) wb.alive[wb.na + __popc(mask & ((1u << lane_id()) - 1u))] = v;
  __syncwarp();
  wb.na += tot;
}

// Append the work items of vertex p (lanes with `push`), stamping it.  All
// lanes call it.  Batches larger than the staging buffer go straight to Q.
__device__ __forceinline__ void push_items(const CoreArgs &a, bool push, int p, WarpBuf &wb,
                                           int4 *Q, unsigned long long *qctr, int stamp_val) {
  const int lane = lane_id();
  int n = 0, L = 0;
  int64_t lb = 0;
  if (push) {
    lb = __ldg(&a.soff[p]);
    L = (int)(__ldg(&a.soff[p + 1]) - lb);
    n = items_of(L);
    a.stamp[p] = stamp_val;
  }
  const int P = warp_incl_scan(n);
  const int tot = __shfl_sync(TR_FULL, P, 31);
  if (tot == 0) return;
  int4 *dst;
  long long b0;
  if (tot > kWQ) {
    unsigned long long b = 0;
    if (lane == 31) b = atomicAdd(qctr, (unsigned long long)tot);
    b0 = (long long)__shfl_sync(TR_FULL, b, 31);
    dst = Q;
  } else {
    if (wb.ni + tot > kWQ) flush_items(a, wb, Q, qctr);
    b0 = wb.ni;
    dst = wb.items;
  }
  const long long lim = tot > kWQ ? a.item_cap : (long long)kWQ;
  for (int t0 = 0; t0 < tot; t0 += 32) {
    const int t = t0 + lane;
    const int o = warp_owner(P, t < tot ? t : tot - 1);
    const int po = __shfl_sync(TR_FULL, p, o);
    const int Po = __shfl_sync(TR_FULL, P, o);
    const int no = __shfl_sync(TR_FULL, n, o);
    const int Lo = __shfl_sync(TR_FULL, L, o);
    const int64_t lbo = __shfl_sync(TR_FULL, lb, o);
    const long long idx = b0 + t;
    if (t < tot && idx < lim) {
      const int it = t - (Po - no);
      const int start = it * kItem;
      const int cnt = Lo > 0 ? min(kItem, Lo - start) : 0;
      const int64_t off = lbo + start;
      dst[idx] = make_int4(po, cnt | ((it == 0) << 8), (int)(uint32_t)off,
                           (int)(uint32_t)((uint64_t)off >> 32));
    }
  }
  __syncwarp();
  if (tot <= kWQ) wb.ni += tot;
}

__global__ void __launch_bounds__(kBlock, 2) k_core(CoreArgs a) {
  const int lane = lane_id();
  const int wib = threadIdx.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * kWarps + wib;
  const int64_t twarps = (int64_t)gridDim.x * kWarps;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  CoreCtl *ctl = a.ctl;
  __shared__ int4 s_items[kWarps][kWQ];
  __shared__ int32_t s_alive[kWarps][kWA];
  __shared__ int s_minres, s_live;
  WarpBuf wb{s_items[wib], 0, s_alive[wib], 0};
  if (threadIdx.x == 0) {
    s_minres = INT_MAX;
    s_live = 0;
  }
  __syncthreads();

  int k = 0, s = 1, sc = 0;
  unsigned ph = 0;
  int32_t *alive = a.alive0, *alive2 = a.alive1;
  int4 *F = a.Q0, *N = a.Q1;
  int64_t nAlive = a.n;
  bool compact = false;

  for (;;) {
    // ------------------------------------------------------------ scan ---
    const int slot = sc % 3;
    unsigned long long *qf = &ctl->qf[ph % 3], *qa = &ctl->qa[ph % 3];
    if (leader) {
      ctl->minres[(sc + 1) % 3] = INT_MAX;
      ctl->live[(sc + 1) % 3] = 0;
      ctl->qf[(ph + 1) % 3] = 0;
      ctl->qa[(ph + 1) % 3] = 0;
    }
    int wmin = INT_MAX, wlive = 0;
    for (int64_t base = gwarp * 32; base < nAlive; base += twarps * 32) {
      const int64_t i = base + lane;
      const int v = i < nAlive ? __ldcg(&alive[i]) : -1;
      const int st = v >= 0 ? __ldcg(&a.stamp[v]) : 1;
      const int dv = v >= 0 ? __ldcg(&a.deg[v]) : 0;
      const bool live = v >= 0 && st == 0;
      const bool toF = live && dv <= k;
      const bool keep = live && !toF;
      push_items(a, toF, v, wb, F, qf, s);
      if (compact) push_alive(a, keep, v, wb, alive2, qa);
      wmin = min(wmin, __reduce_min_sync(TR_FULL, keep ? dv : INT_MAX));
      wlive += __popc(__ballot_sync(TR_FULL, keep));
    }
    flush_items(a, wb, F, qf);
    if (compact) flush_alive(a, wb, alive2, qa);
    if (lane == 0) {
      if (wmin != INT_MAX) atomicMin(&s_minres, wmin);
      if (wlive) atomicAdd(&s_live, wlive);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_minres != INT_MAX) atomicMin(&ctl->minres[slot], s_minres);
      if (s_live) atomicAdd(&ctl->live[slot], s_live);
      s_minres = INT_MAX;
      s_live = 0;
    }
    if (!grid_barrier(&ctl->bar, &ctl->err, a.wait_ns)) return;
    ph++;
    const int minres = __ldcg(&ctl->minres[slot]);
    const int64_t live = __ldcg(&ctl->live[slot]);
    const int64_t nF = (int64_t)__ldcg(qf);
    if (compact) {
      nAlive = (int64_t)__ldcg(qa);
      int32_t *t = alive;
      alive = alive2;
      alive2 = t;
    }
    compact = 2 * live <= nAlive;
    sc++;
    if (nF == 0) {
      if (live == 0) break;
      k = minres;  // every alive vertex has degree >= k+1: skip empty levels
      continue;
    }
    // --------------------------------------------------------- sub-rounds ---
    int64_t nCur = nF > a.item_cap ? a.item_cap : nF;
    if (nF > a.item_cap && leader) atomicExch(&ctl->err, TRUSS_ECHECK);
    for (;;) {
      unsigned long long *qn = &ctl->qf[ph % 3];
      if (leader) {
        ctl->qf[(ph + 1) % 3] = 0;
        ctl->qa[(ph + 1) % 3] = 0;
      }
      const int grp = lane >> 3, j = lane & 7;
      for (int64_t base = gwarp * 4; base < nCur; base += twarps * 4) {
        const int64_t it = base + grp;
        int v = 0, cnt = 0;
        int64_t lb = 0;
        if (it < nCur) {
          const int4 item = __ldcg(&F[it]);
          v = item.x;
          cnt = item.y & 0xFF;
          lb = (int64_t)(((uint64_t)(uint32_t)item.w << 32) | (uint32_t)item.z);
          if ((item.y >> 8) && j == 0) a.core[v] = k;
        }
        int w[2];
        bool dec[2];
#pragma unroll
        for (int q = 0; q < 2; q++) {
          const int jj = j + 8 * q;
          w[q] = jj < cnt ? __ldg(&a.sadj[lb + jj]) : -1;
        }
#pragma unroll
        for (int q = 0; q < 2; q++) {
          dec[q] = false;
          if (w[q] >= 0) {
            if ((uint32_t)w[q] >= (uint32_t)a.n) {
              atomicExch(&ctl->err, TRUSS_ECHECK);
            } else {
              const int sw = __ldcg(&a.stamp[w[q]]);
              dec[q] = sw == 0 || sw > s;  // alive (possibly pushed this sub-round)
            }
          }
        }
        int old[2];
#pragma unroll
        for (int q = 0; q < 2; q++) old[q] = dec[q] ? atomicSub(&a.deg[w[q]], 1) : INT_MIN;
        // one push_items site: each step pushes one pending neighbour per lane
        unsigned pend = (old[0] == k + 1 ? 1u : 0u) | (old[1] == k + 1 ? 2u : 0u);
        while (__any_sync(TR_FULL, pend != 0)) {
          const bool has = pend != 0;
          const int b = has ? __ffs(pend) - 1 : 0;
          pend &= pend - 1;
          push_items(a, has, b ? w[1] : w[0], wb, N, qn, s + 1);
        }
      }
      flush_items(a, wb, N, qn);
      if (!grid_barrier(&ctl->bar, &ctl->err, a.wait_ns)) return;
      ph++;
      const int64_t nN = (int64_t)__ldcg(qn);
      s++;
      if (leader) ctl->subrounds++;
      if (nN == 0) break;
      { int4 *t = F; F = N; N = t; }
      nCur = nN > a.item_cap ? a.item_cap : nN;
      if (nN > a.item_cap && leader) atomicExch(&ctl->err, TRUSS_ECHECK);
    }
    if (leader) {
      ctl->levels++;
      ctl->kmax = k;
    }
    k++;
  }
}

// Symmetric degrees: out-degree plus in-degree of every vertex.
__global__ void k_sym_deg(int64_t n, int64_t m, const int64_t *offp, const int32_t *adjp,
                          unsigned long long *sdeg) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&sdeg[adjp[e]], 1ull);
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&sdeg[v], (unsigned long long)(offp[v + 1] - offp[v]));
}

// sadj[soff[v] ..) = all neighbours of v, in any order.
__global__ void k_sym_fill(int64_t m, const int32_t *esrc, const int32_t *adjp,
                           const int64_t *soff, unsigned long long *cur, int32_t *sadj) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int u = esrc[e], v = adjp[e];
    sadj[soff[u] + (int64_t)atomicAdd(&cur[u], 1ull)] = v;
    sadj[soff[v] + (int64_t)atomicAdd(&cur[v], 1ull)] = u;
  }
}

__global__ void k_core_init(int64_t n, const int64_t *soff, int32_t *deg, int32_t *stamp,
                            int32_t *alive, CoreCtl *ctl) {
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->minres[0] = INT_MAX;  // first scan's slot
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    deg[v] = (int32_t)(soff[v + 1] - soff[v]);
    stamp[v] = 0;
    alive[v] = (int32_t)v;
  }
}

// core_out[order[r]] = core[r]: back from ranks to input vertex ids.
__global__ void k_core_out(int64_t n, const int32_t *order, const int32_t *core,
                           int32_t *core_out) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    core_out[order[r]] = core[r];
}

}  // namespace

int run_core(Arena &A, const Csr &g, int sms, long long wait_ns, int32_t *core_out,
             int32_t *kmax, int32_t *levels, int32_t *subrounds, cudaStream_t s) {
  const int64_t n = g.n, m = g.m;
  *kmax = 0;
  *levels = *subrounds = 0;
  if (n == 0) return TRUSS_OK;
  unsigned long long *cnt = A.get<unsigned long long>(n + 1);
  int64_t *soff = A.get<int64_t>(n + 1);
  int32_t *sadj = A.get<int32_t>(2 * m);
  int32_t *deg = A.get<int32_t>(n), *stamp = A.get<int32_t>(n), *core = A.get<int32_t>(n);
  int32_t *al0 = A.get<int32_t>(n), *al1 = A.get<int32_t>(n);
  // every vertex is pushed at most once; its items number at most
  // deg / kItem + 1, so 2m / kItem + n items bound any frontier
  const int64_t item_cap = 2 * m / kItem + n + 1;
  int4 *Q0 = A.get<int4>(item_cap), *Q1 = A.get<int4>(item_cap);
  CoreCtl *ctl = A.get<CoreCtl>(1);
  if (!cnt || !soff || !sadj || !deg || !stamp || !core || !al0 || !al1 || !Q0 || !Q1 || !ctl)
    return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (n + 1), s));
  k_sym_deg<<<grid_for(m > n ? m : n, 256, 152 * 16), 256, 0, s>>>(n, m, g.offp, g.adjp, cnt);
  TR_LAUNCHED();
  size_t tb = 0;
  TR_TRY(exclusive_sum_i64(nullptr, &tb, (const int64_t *)cnt, soff, n + 1, s));
  void *tmp = A.alloc(tb);
  if (!tmp) return TRUSS_ENOMEM;
  TR_TRY(exclusive_sum_i64(tmp, &tb, (const int64_t *)cnt, soff, n + 1, s));
  TR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (n + 1), s));
  if (m > 0) {
    k_sym_fill<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, g.esrc, g.adjp, soff, cnt, sadj);
    TR_LAUNCHED();
  }
  TR_CUDA(cudaMemsetAsync(ctl, 0, sizeof(CoreCtl), s));
  k_core_init<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(n, soff, deg, stamp, al0, ctl);
  TR_LAUNCHED();
  int occ = 0;
  TR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_core, kBlock, 0));
  if (occ < 1) return TRUSS_ECUDA;
  if (occ > 2) occ = 2;
  CoreArgs a{};
  a.n = n;
  a.soff = soff;
  a.sadj = sadj;
  a.deg = deg;
  a.stamp = stamp;
  a.core = core;
  a.alive0 = al0;
  a.alive1 = al1;
  a.Q0 = Q0;
  a.Q1 = Q1;
  a.item_cap = item_cap;
  a.ctl = ctl;
  a.wait_ns = wait_ns;
  void *args[] = {&a};
  TR_CUDA(cudaLaunchCooperativeKernel((const void *)k_core, dim3(sms * occ), dim3(kBlock), args,
                                      0, s));
  count_launches(1);
  k_core_out<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(n, g.order, core, core_out);
  TR_LAUNCHED();
  CoreCtl h{};
  TR_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(CoreCtl), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  if (h.err != 0) return h.err;
  *kmax = h.kmax;
  *levels = h.levels;
  *subrounds = h.subrounds;
  return TRUSS_OK;
}

}  // namespace tr
