// Edge peeling without sub-round barriers (Algorithm 2 steps 3-16, exact).
//
// The level-synchronous peel (peel.cu) needs a grid barrier after every
// sub-round so that all blocks agree on which edges are in the frontier
// when they decide who charges a triangle.  Here each triangle carries a
// "destroyed" bit instead (its record index, written next to every list
// entry by the list passes): the first removed edge that sets the bit
// charges the triangle, decrementing its two other edges once, whatever the
// order in which concurrent removals reach it.  Then no frontier needs to be
// agreed on, and inside a level the removals run as a work queue:
//
//  scan (level k, one grid barrier):  alive edges with res <= k-2 are
//        removed (truss k) and queued; the minimum residual of the rest lets
//        an empty level jump ahead.
//  drain:  warps take queued items (kItem list entries of one removed edge),
//        never past the queued count, and wait for each item's ready flag.  For each triangle whose bit they set, both
//        partners lose one residual; a partner whose residual crosses
//        k-1 -> k-2 and that is still alive (claimed with a compare-and-swap
//        on its stamp) is removed with truss k and its items are queued.
//        The level ends when every queued item is done: reading the done
//        count first and the queued count second, equal values mean that
//        nothing was in flight, so nothing can be queued any more.
//
// Why exact: res(e) of an alive edge counts its triangles not yet destroyed,
// which include every triangle of alive edges only; an edge removed at level
// k had at most k-2 such triangles when it was claimed, so it is not in
// T_{k+1}; and once the level drains, every alive edge has res >= k-1 over
// triangles whose three edges are alive, so the alive edges form a
// subgraph inside T_{k+1}.  So the removed set of each level is T_k \ T_{k+1}.
//
// The queue is one array for the whole run (every edge is queued once),
// with a ready flag per slot written after the item; counters are monotone.
// Every wait is bounded by wait_ns (TRUSS_ETIMEOUT).
#include <climits>

#include "engine.h"

namespace tr {

namespace {

constexpr int kBlock = 512;
constexpr int kWarps = kBlock / 32;
constexpr int kItem = 16;  // list entries per work item (8 lanes x 2)
constexpr int kWA = 128;   // alive-list entries staged per warp

struct AsyncCtl {
  unsigned long long bar;
  int err;
  int pad0;
  unsigned long long tail;  // items queued (whole run)
  unsigned long long head;  // items taken
  unsigned long long done;  // items finished
  unsigned long long qa[3]; // alive-list entries appended in scan s (slot s % 3)
  unsigned long long qs[3]; // items queued by scan s (slot s % 3)
  int minres[3];
  int live[3];
  int levels, kmax, pad1, pad2;
  unsigned long long entries, decrements, scanned;
};

struct AsyncArgs {
  int64_t m;
  const int64_t *toff;
  const int32_t *sup;
  const int2 *pairs;
  const uint32_t *tids;  // triangle (record) index of each list entry
  unsigned *dbits;       // destroyed bit per triangle
  int64_t ntri;          // triangle ids are below this
  int32_t *res, *stamp, *truss;
  int32_t *alive0, *alive1;
  int4 *Q;
  unsigned *ready;  // per queue slot: 1 once the item is written
  int64_t item_cap;
  AsyncCtl *ctl;
  long long wait_ns;
};

__device__ __forceinline__ int items_of(int len) { return len > 0 ? (len + kItem - 1) / kItem : 1; }

// Queue the items of edge p for the lanes with `push` (all lanes call it):
// one reservation per warp, the items, then their ready flags.
__device__ __forceinline__ int queue_items(const AsyncArgs &a, bool push, int p) {
  const int lane = lane_id();
  int n = 0, L = 0;
  int64_t lb = 0;
  if (push) {
    L = __ldg(&a.sup[p]);
    lb = __ldg(&a.toff[p]);
    n = items_of(L);
  }
  const int P = warp_incl_scan(n);
  const int tot = __shfl_sync(TR_FULL, P, 31);
  if (tot == 0) return 0;
  unsigned long long b = 0;
  if (lane == 31) b = atomicAdd(&a.ctl->tail, (unsigned long long)tot);
  const long long b0 = (long long)__shfl_sync(TR_FULL, b, 31);
  for (int t0 = 0; t0 < tot; t0 += 32) {
    const int t = t0 + lane;
    const int o = warp_owner(P, t < tot ? t : tot - 1);
    const int po = __shfl_sync(TR_FULL, p, o);
    const int Po = __shfl_sync(TR_FULL, P, o);
    const int no = __shfl_sync(TR_FULL, n, o);
    const int Lo = __shfl_sync(TR_FULL, L, o);
    const int64_t lbo = __shfl_sync(TR_FULL, lb, o);
    const long long idx = b0 + t;
    if (t < tot && idx < a.item_cap) {
      const int it = t - (Po - no);
      const int start = it * kItem;
      const int cnt = Lo > 0 ? min(kItem, Lo - start) : 0;
      const int64_t off = lbo + start;
      a.Q[idx] = make_int4(po, cnt, (int)(uint32_t)off, (int)(uint32_t)((uint64_t)off >> 32));
    } else if (t < tot) {
      atomicExch(&a.ctl->err, TRUSS_ECHECK);
    }
  }
  __threadfence();
  for (int t = lane; t < tot; t += 32)
    if (b0 + t < a.item_cap) atomicExch(&a.ready[b0 + t], 1u);
  return tot;
}

__device__ __forceinline__ void flush_alive(const AsyncArgs &a, int32_t *wbuf, int &na,
                                            int32_t *A2, unsigned long long *actr) {
  if (na == 0) return;
  const int lane = lane_id();
  unsigned long long b = 0;
  if (lane == 0) b = atomicAdd(actr, (unsigned long long)na);
  const long long b0 = (long long)__shfl_sync(TR_FULL, b, 0);
  for (int t = lane; t < na; t += 32)
    if (b0 + t < a.m) A2[b0 + t] = wbuf[t];
  __syncwarp();
  na = 0;
}

__global__ void __launch_bounds__(kBlock, 2) k_peel_async(AsyncArgs a) {
  const int lane = lane_id();
  const int wib = threadIdx.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * kWarps + wib;
  const int64_t twarps = (int64_t)gridDim.x * kWarps;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  AsyncCtl *ctl = a.ctl;
  __shared__ int32_t s_alive[kWarps][kWA];
  __shared__ int s_minres, s_live;
  __shared__ unsigned long long s_queued;
  int32_t *wbuf = s_alive[wib];
  int na = 0;
  if (threadIdx.x == 0) {
    s_minres = INT_MAX;
    s_live = 0;
    s_queued = 0;
  }
  __syncthreads();
  int k = 2, sc = 0;
  int32_t *alive = a.alive0, *alive2 = a.alive1;
  int64_t nAlive = a.m;
  bool compact = false;
  unsigned long long tq = 0;  // queue length when the last level drained
  unsigned long long n_ent = 0, n_dec = 0, n_scan = 0;

  for (;;) {
    // ------------------------------------------------------------ scan ---
    const int slot = sc % 3;
    unsigned long long *qa = &ctl->qa[slot];
    if (leader) {
      ctl->minres[(sc + 1) % 3] = INT_MAX;
      ctl->live[(sc + 1) % 3] = 0;
      ctl->qa[(sc + 1) % 3] = 0;
      ctl->qs[(sc + 1) % 3] = 0;
      ctl->head = tq;  // slots taken past the drained queue are given back
    }
    int wmin = INT_MAX, wlive = 0;
    unsigned long long wq = 0;
    for (int64_t base = gwarp * 32; base < nAlive; base += twarps * 32) {
      const int64_t i = base + lane;
      const int e = i < nAlive ? __ldcg(&alive[i]) : -1;
      const int st = e >= 0 ? __ldcg(&a.stamp[e]) : 1;
      const int r = e >= 0 ? __ldcg(&a.res[e]) : 0;
      const bool live = e >= 0 && st == 0;
      const bool rem = live && r <= k - 2;
      const bool keep = live && !rem;
      if (rem) {
        a.stamp[e] = 1;
        a.truss[e] = k;
      }
      wq += (unsigned long long)queue_items(a, rem, e);
      if (compact) {
        const unsigned mask = __ballot_sync(TR_FULL, keep);
        const int tot = __popc(mask);
        if (tot) {
          if (na + tot > kWA) flush_alive(a, wbuf, na, alive2, qa);
          if (keep) wbuf[na + __popc(mask & ((1u << lane) - 1u))] = e;
          __syncwarp();
          na += tot;
        }
      }
      wmin = min(wmin, __reduce_min_sync(TR_FULL, keep ? r : INT_MAX));
      wlive += __popc(__ballot_sync(TR_FULL, keep));
      n_scan += (e >= 0);
    }
    if (compact) flush_alive(a, wbuf, na, alive2, qa);
    if (lane == 0) {
      if (wmin != INT_MAX) atomicMin(&s_minres, wmin);
      if (wlive) atomicAdd(&s_live, wlive);
      if (wq) atomicAdd(&s_queued, wq);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (s_minres != INT_MAX) atomicMin(&ctl->minres[slot], s_minres);
      if (s_live) atomicAdd(&ctl->live[slot], s_live);
      if (s_queued) atomicAdd(&ctl->qs[slot], s_queued);
      s_minres = INT_MAX;
      s_live = 0;
      s_queued = 0;
    }
    if (!grid_barrier(&ctl->bar, &ctl->err, a.wait_ns)) return;
    const int minres = __ldcg(&ctl->minres[slot]);
    const int64_t live = __ldcg(&ctl->live[slot]);
    // the scan's own count: the shared tail may already hold the next scan's
    // items of blocks that left this barrier first
    const unsigned long long nq = __ldcg(&ctl->qs[slot]);
    if (compact) {
      nAlive = (int64_t)__ldcg(qa);
      int32_t *t = alive;
      alive = alive2;
      alive2 = t;
    }
    compact = 2 * live <= nAlive;
    sc++;
    if (nq == 0) {  // nothing removed at this level
      if (live == 0) break;
      k = minres + 2;
      continue;
    }
    // ------------------------------------------------------------ drain ---
    const int grp = lane >> 3, j = lane & 7;
    const unsigned long long t0 = global_ns();
    int spins = 0;
    // each 8-lane group holds one queue slot at a time; a slot taken past the
    // queued count waits until a warp queues an item there, or the level
    // drains (then the next scan gives it back by resetting head)
    unsigned long long mine = ~0ull;
    for (;;) {
      const bool need = mine == ~0ull;
      const unsigned nmask = __ballot_sync(TR_FULL, need && j == 0);
      if (nmask) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(&ctl->head, (unsigned long long)__popc(nmask));
        b = __shfl_sync(TR_FULL, b, 0);
        if (need) mine = b + (unsigned long long)__popc(nmask & ((1u << (grp * 8)) - 1u));
      }
      // one lane per group reads the flag, so the group's lanes agree
      bool rdy = false;
      if (j == 0) rdy = mine < (unsigned long long)a.item_cap &&
                        *(volatile unsigned *)&a.ready[mine] != 0u;
      const bool have = __shfl_sync(TR_FULL, rdy, lane & ~7);
      const unsigned hmask = __ballot_sync(TR_FULL, have && j == 0);
      if (hmask == 0) {
        // nothing ready: drained?  done first, then tail: equal means nothing
        // was in flight, so nothing can be queued any more
        unsigned long long d = 0, t = 0;
        if (lane == 0) {
          d = *(volatile unsigned long long *)&ctl->done;
          __threadfence();
          t = *(volatile unsigned long long *)&ctl->tail;
        }
        d = __shfl_sync(TR_FULL, d, 0);
        t = __shfl_sync(TR_FULL, t, 0);
        if (d == t) {
          tq = t;
          break;
        }
        if (++spins > 16) __nanosleep(64);
        bool late = false;
        if (lane == 0) late = (long long)(global_ns() - t0) > a.wait_ns;
        if (__shfl_sync(TR_FULL, late, 0)) {
          if (lane == 0) atomicExch(&ctl->err, TRUSS_ETIMEOUT);
          break;
        }
        if (*(volatile int *)&ctl->err != 0) break;
        continue;
      }
      spins = 0;
      __threadfence();
      int e = 0, cnt = 0;
      int64_t lb = 0;
      if (have) {
        const int4 item = __ldcg(&a.Q[mine]);
        e = item.x;
        cnt = item.y;
        lb = (int64_t)(((uint64_t)(uint32_t)item.w << 32) | (uint32_t)item.z);
        if (__ldcg(&a.res[e]) == 0) cnt = 0;  // all of e's triangles are gone
      }
      int2 pp[2];
      uint32_t tid[2];
      bool v[2];
#pragma unroll
      for (int q = 0; q < 2; q++) {
        const int jj = j + 8 * q;
        v[q] = have && jj < cnt;
        pp[q] = v[q] ? __ldcs(&a.pairs[lb + jj]) : make_int2(0, 0);
        tid[q] = v[q] ? __ldcs(&a.tids[lb + jj]) : 0u;
      }
      bool chg[2];
#pragma unroll
      for (int q = 0; q < 2; q++) {
        chg[q] = false;
        if (v[q]) {
          if ((uint32_t)pp[q].x >= (uint32_t)a.m || (uint32_t)pp[q].y >= (uint32_t)a.m ||
              (int64_t)tid[q] >= a.ntri) {
            atomicExch(&ctl->err, TRUSS_ECHECK);
          } else {
            const unsigned bit = 1u << (tid[q] & 31u);
            chg[q] = (atomicOr(&a.dbits[tid[q] >> 5], bit) & bit) == 0u;
          }
          n_ent++;
        }
      }
      int o[4];
#pragma unroll
      for (int q = 0; q < 2; q++) {
        o[2 * q] = chg[q] ? atomicSub(&a.res[pp[q].x], 1) : INT_MAX;
        o[2 * q + 1] = chg[q] ? atomicSub(&a.res[pp[q].y], 1) : INT_MAX;
        n_dec += chg[q] ? 2 : 0;
      }
      bool claim[4];
      int pe[4] = {pp[0].x, pp[0].y, pp[1].x, pp[1].y};
#pragma unroll
      for (int q = 0; q < 4; q++) {
        claim[q] = o[q] == k - 1 && atomicCAS(&a.stamp[pe[q]], 0, 1) == 0;
        if (claim[q]) a.truss[pe[q]] = k;
      }
      if (__any_sync(TR_FULL, claim[0] || claim[1] || claim[2] || claim[3])) {
#pragma unroll
        for (int q = 0; q < 4; q++) (void)queue_items(a, claim[q], pe[q]);
      }
      // this warp's items are finished (their children are already queued)
      __threadfence();
      if (lane == 0) atomicAdd(&ctl->done, (unsigned long long)__popc(hmask));
      if (have) mine = ~0ull;
    }
    if (!grid_barrier(&ctl->bar, &ctl->err, a.wait_ns)) return;
    if (leader) {
      ctl->levels++;
      ctl->kmax = k;
    }
    k++;
  }
  for (int o = 16; o >= 1; o >>= 1) {
    n_ent += __shfl_down_sync(TR_FULL, n_ent, o);
    n_dec += __shfl_down_sync(TR_FULL, n_dec, o);
    n_scan += __shfl_down_sync(TR_FULL, n_scan, o);
  }
  if (lane == 0) {
    atomicAdd(&ctl->entries, n_ent);
    atomicAdd(&ctl->decrements, n_dec);
    atomicAdd(&ctl->scanned, n_scan);
  }
}

__global__ void k_async_init(int64_t m, const int32_t *sup, int32_t *res, int32_t *stamp,
                             int32_t *alive, int32_t *truss, AsyncCtl *ctl) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    res[e] = sup[e];
    stamp[e] = 0;
    alive[e] = (int32_t)e;
    truss[e] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int i = 0; i < 3; i++) {
      ctl->minres[i] = INT_MAX;
      ctl->live[i] = 0;
    }
}

}  // namespace

int run_peel_async(Arena &A, const Csr &g, const SupportOut &so, const int2 *pairs,
                   const uint32_t *tids, int64_t ntri, const PeelCfg &cfg, int32_t *truss,
                   PeelResult *out, cudaStream_t s) {
  const int64_t m = g.m;
  *out = PeelResult{};
  if (m == 0) return TRUSS_OK;
  // every edge is queued once: at most max(1, ceil(sup / kItem)) items each
  const int64_t item_cap = m + so.entries / kItem + 64;
  const int64_t words = (ntri + 31) / 32 + 1;
  int32_t *res = A.get<int32_t>(m), *stamp = A.get<int32_t>(m);
  int32_t *al0 = A.get<int32_t>(m), *al1 = A.get<int32_t>(m);
  int4 *Q = A.get<int4>(item_cap);
  unsigned *ready = A.get<unsigned>(item_cap), *dbits = A.get<unsigned>(words);
  AsyncCtl *ctl = A.get<AsyncCtl>(1);
  if (!res || !stamp || !al0 || !al1 || !Q || !ready || !dbits || !ctl) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(ctl, 0, sizeof(AsyncCtl), s));
  TR_CUDA(cudaMemsetAsync(ready, 0, sizeof(unsigned) * item_cap, s));
  TR_CUDA(cudaMemsetAsync(dbits, 0, sizeof(unsigned) * words, s));
  k_async_init<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, so.sup, res, stamp, al0, truss, ctl);
  TR_LAUNCHED();
  int dev = 0, sms = cfg.sms;
  TR_CUDA(cudaGetDevice(&dev));
  if (sms <= 0) TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int occ = 0;
  TR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peel_async, kBlock, 0));
  if (occ < 1) return TRUSS_ECUDA;
  if (occ > 2) occ = 2;
  AsyncArgs a{};
  a.m = m;
  a.toff = so.toff;
  a.sup = so.sup;
  a.pairs = pairs;
  a.tids = tids;
  a.dbits = dbits;
  a.ntri = ntri;
  a.res = res;
  a.stamp = stamp;
  a.truss = truss;
  a.alive0 = al0;
  a.alive1 = al1;
  a.Q = Q;
  a.ready = ready;
  a.item_cap = item_cap;
  a.ctl = ctl;
  a.wait_ns = cfg.wait_ns;
  void *args[] = {&a};
  TR_CUDA(cudaLaunchCooperativeKernel((const void *)k_peel_async, dim3(sms * occ), dim3(kBlock),
                                      args, 0, s));
  count_launches(1);
  AsyncCtl h{};
  TR_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(AsyncCtl), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  out->err = h.err;
  out->kmax = h.kmax;
  out->levels = h.levels;
  out->subrounds = 0;
  out->entries = h.entries;
  out->decrements = h.decrements;
  out->scanned = h.scanned;
  if (h.err != 0) return h.err;
  return TRUSS_OK;
}

}  // namespace tr
