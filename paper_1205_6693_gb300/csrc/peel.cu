// Level-synchronous edge peeling (Algorithm 2 steps 3-16) in one persistent
// cooperative launch.
//
// Algorithm 2 removes, for k = 2, 3, ..., the lowest-support edge while its
// support is <= k-2, decrementing the support of the other two edges of each
// triangle it destroys (steps 7-10) and assigning it to Phi_k (step 11).  The
// order in which edges of one level are removed does not change the result
// (T_k is unique, Definition 2), so here every level is processed in
// sub-rounds: all alive edges whose residual support res is <= k-2 form the
// frontier F and are removed together.
//
//  scan (per level k):  F = {alive e : res[e] <= k-2}; the other alive edges
//        are compacted into the next alive list and their minimum residual
//        is taken, so an empty level jumps straight to k = min res + 2.
//  sub-round:  for every e in F and every triangle {e, e1, e2} on e's list
//        whose edges are all still alive, the triangle is charged exactly
//        once, by the lowest-id edge among those of its edges that are in F:
//        that edge decrements the residual of each partner not in F.  A
//        partner whose residual crosses from k-1 to k-2 joins the next
//        frontier (warp-aggregated append).  F edges get truss number k.
//
// Load balance inside a sub-round (its time is that of the slowest warp):
// when an edge joins a frontier it is expanded into work items of kItem list
// entries each (at least one item, which also records its truss number), and
// every warp takes 4 items per iteration, 8 lanes per item.  A warp's share of
// a sub-round is then at most ceil(items / (4 * warps)) iterations, whatever
// the lengths of the lists.
// The queues use monotonically increasing 64-bit counters (never reset).  The
// block that completes a grid barrier copies them into a snapshot slot of
// that barrier's generation before releasing it, and every block takes its
// next bases from the snapshot: a block that leaves the barrier early may
// already append to the live counters while a slow one has not read them.
//
// Edge state is one int per edge, stamp[e]: 0 = alive, s = in the frontier of
// sub-round s, 0 < stamp < s = removed earlier.  A partner pushed during
// sub-round s is stamped s+1, which reads as alive during s, so one grid
// barrier per sub-round suffices.  res[e] of a frontier edge is never touched
// during its sub-round and equals the number of its still-alive triangles,
// so a frontier edge with res 0 skips its list.
//
// Every grid barrier waits at most `wait_ns` (globaltimer); on timeout the
// kernel records TRUSS_ETIMEOUT and all blocks return at their next barrier.
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "engine.h"

namespace tr {

namespace {

constexpr int kPeelBlock = 512;
constexpr int kItem = 8;  // list entries per work item (one lane each)

struct PeelCtl {
  unsigned bar_count;
  unsigned bar_gen;
  int err;
  int pad0;
  unsigned long long qf;  // frontier items appended so far (F and N alternate)
  unsigned long long qa;  // alive-list entries appended so far
  int minres[3];          // per scan phase (slot = scan index % 3)
  int pad1;
  unsigned long long snap[2][2];  // qf, qa at the last two barriers
  int levels, subrounds, kmax, pad2;
  unsigned long long entries, decrements, scanned;
};

struct PeelArgs {
  int64_t m;
  const int64_t *toff;
  const int32_t *sup;
  const int2 *pairs;
  int32_t *res;
  int32_t *stamp;
  int32_t *truss;
  int32_t *alive0, *alive1;
  int2 *Q0, *Q1;      // frontier work items (edge, item index)
  int64_t item_cap;   // capacity of Q0 and Q1
  int4 *trace;        // optional: per sub-round (k, items, 0, 0)
  int trace_cap;
  PeelCtl *ctl;
  long long wait_ns;
};

// Grid-wide barrier with a time limit.  On return every thread of the block
// sees in `snap` the values of qf and qa at the moment the last block
// arrived.  Returns false if any block has recorded an error (including this
// barrier timing out).
__device__ bool grid_barrier(PeelCtl *c, long long wait_ns, unsigned long long *snap) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = &c->bar_gen;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      __threadfence();
      volatile unsigned long long *sn = c->snap[g & 1];
      sn[0] = __ldcg(&c->qf);
      sn[1] = __ldcg(&c->qa);
      atomicExch(&c->bar_count, 0u);
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      int spins = 0;
      while (*vgen == g) {
        if (++spins > 64) __nanosleep(64);
        if ((long long)(global_ns() - t0) > wait_ns) {
          atomicExch(&c->err, TRUSS_ETIMEOUT);
          break;
        }
      }
    }
    __threadfence();
    volatile unsigned long long *sn = c->snap[g & 1];
    snap[0] = sn[0];
    snap[1] = sn[1];
    s_ok = (*(volatile int *)&c->err) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ int items_of(int len) { return len > 0 ? (len + kItem - 1) / kItem : 1; }

// Append the work items of edge p (for each lane with `push`) to queue Q,
// stamping p with `stamp_val`.  All lanes call it.
__device__ __forceinline__ void push_items(const PeelArgs &a, bool push, int p, int2 *Q,
                                           unsigned long long base_q, int stamp_val) {
  const int lane = lane_id();
  int n = 0;
  if (push) {
    n = items_of(__ldg(&a.sup[p]));
    a.stamp[p] = stamp_val;
  }
  const int P = warp_incl_scan(n);
  const int tot = __shfl_sync(TR_FULL, P, 31);
  if (tot == 0) return;
  unsigned long long b = 0;
  if (lane == 31) b = atomicAdd(&a.ctl->qf, (unsigned long long)tot);
  const long long b0 = (long long)(__shfl_sync(TR_FULL, b, 31) - base_q);
  for (int t0 = 0; t0 < tot; t0 += 32) {
    const int t = t0 + lane;
    const int o = warp_owner(P, t < tot ? t : tot - 1);
    const int po = __shfl_sync(TR_FULL, p, o);
    const int Po = __shfl_sync(TR_FULL, P, o);
    const int no = __shfl_sync(TR_FULL, n, o);
    const long long idx = b0 + t;
    if (t < tot && idx < a.item_cap) Q[idx] = make_int2(po, t - (Po - no));
  }
}

// One triangle entry (the partner edges p1, p2 of frontier edge e) in
// sub-round s at level k; all lanes call it (`valid` masks idle lanes).
// Charges the triangle by the lowest-id frontier edge among its edges and
// appends partners whose residual crosses k-1 -> k-2 to the next frontier.
__device__ __forceinline__ void charge(const PeelArgs &a, bool valid, int e, int2 pr, int k,
                                       int s, int2 *N, unsigned long long base_f,
                                       unsigned long long &n_dec) {
  bool d1 = false, d2 = false;
  const int p1 = pr.x, p2 = pr.y;
  if (valid) {
    if ((uint32_t)p1 >= (uint32_t)a.m || (uint32_t)p2 >= (uint32_t)a.m) {
      atomicExch(&a.ctl->err, TRUSS_ECHECK);  // corrupt list entry: skip it
    } else {
      const int s1 = __ldcg(&a.stamp[p1]), s2 = __ldcg(&a.stamp[p2]);
      const bool dead1 = s1 > 0 && s1 < s, dead2 = s2 > 0 && s2 < s;
      if (!dead1 && !dead2) {
        const bool in1 = s1 == s, in2 = s2 == s;
        if (!in1 && !in2) {
          d1 = true;
          d2 = true;
        } else if (in1 && !in2) {
          d2 = e < p1;  // e and e1 in F: the lower id charges e2
        } else if (!in1 && in2) {
          d1 = e < p2;
        }
      }
    }
  }
  bool push1 = false, push2 = false;
  if (d1) push1 = atomicSub(&a.res[p1], 1) == k - 1;
  if (d2) push2 = atomicSub(&a.res[p2], 1) == k - 1;
  n_dec += (unsigned long long)(d1 + d2);
  if (__any_sync(TR_FULL, push1 || push2)) {
    push_items(a, push1, p1, N, base_f, s + 1);
    push_items(a, push2, p2, N, base_f, s + 1);
  }
}

__global__ void __launch_bounds__(kPeelBlock) k_peel(PeelArgs a) {
  const int lane = lane_id();
  const int nw = blockDim.x >> 5;
  const int64_t gwarp = (int64_t)blockIdx.x * nw + (threadIdx.x >> 5);
  const int64_t twarps = (int64_t)gridDim.x * nw;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  PeelCtl *ctl = a.ctl;
  __shared__ unsigned long long snap[2];  // qf, qa at the last barrier

  int k = 2, s = 1, sc = 0;
  unsigned long long base_f = 0, base_a = 0;
  int32_t *alive = a.alive0, *alive2 = a.alive1;
  int2 *F = a.Q0, *N = a.Q1;
  int64_t nAlive = a.m;
  unsigned long long n_entries = 0, n_dec = 0, n_scan = 0;

  for (;;) {
    // ------------------------------------------------------------ scan ---
    int *mres = &ctl->minres[sc % 3];
    if (leader) ctl->minres[(sc + 1) % 3] = INT_MAX;
    for (int64_t base = gwarp * 32; base < nAlive; base += twarps * 32) {
      const int64_t i = base + lane;
      int e = -1, r = 0;
      bool live = false;
      if (i < nAlive) {
        e = __ldcg(&alive[i]);
        if (__ldcg(&a.stamp[e]) == 0) {
          live = true;
          r = __ldcg(&a.res[e]);
        }
      }
      const bool toF = live && r <= k - 2;
      const bool keep = live && !toF;
      push_items(a, toF, e, F, base_f, s);
      const long long pa = warp_append64(keep, &ctl->qa);
      if (keep) alive2[pa - (long long)base_a] = e;
      const int mr = __reduce_min_sync(TR_FULL, keep ? r : INT_MAX);
      if (lane == 0 && mr != INT_MAX) atomicMin(mres, mr);
      n_scan += (i < nAlive);
    }
    if (!grid_barrier(ctl, a.wait_ns, snap)) return;
    const int minres = __ldcg(mres);
    const int64_t nF = (int64_t)(snap[0] - base_f), nA = (int64_t)(snap[1] - base_a);
    base_f = snap[0];
    base_a = snap[1];
    sc++;
    { int32_t *t = alive; alive = alive2; alive2 = t; }
    nAlive = nA;
    if (nF == 0) {
      if (nA == 0) break;
      k = minres + 2;  // every alive edge has res >= k-1: skip empty levels
      continue;
    }
    // --------------------------------------------------------- sub-rounds ---
    int64_t nCur = nF;
    for (;;) {
      if (leader && a.trace && ctl->subrounds < a.trace_cap)
        a.trace[ctl->subrounds] = make_int4(k, (int)min(nCur, (int64_t)INT_MAX), 0, 0);
      const int grp = lane >> 3, j = lane & (kItem - 1);
      for (int64_t base = gwarp * 4; base < nCur; base += twarps * 4) {
        const int64_t it = base + grp;
        int e = 0, cnt = 0;
        int64_t lb = 0;
        if (it < nCur) {
          const int2 item = __ldcg(&F[it]);
          e = item.x;
          const int start = item.y * kItem;
          if (item.y == 0 && j == 0) a.truss[e] = k;
          if (__ldcg(&a.res[e]) > 0) {
            cnt = min(kItem, __ldg(&a.sup[e]) - start);
            lb = __ldg(&a.toff[e]) + start;
          }
        }
        const bool valid = j < cnt;
        int2 pr = make_int2(0, 0);
        if (valid) pr = __ldg(&a.pairs[lb + j]);
        n_entries += valid ? 1ull : 0ull;
        charge(a, valid, e, pr, k, s, N, base_f, n_dec);
      }
      if (!grid_barrier(ctl, a.wait_ns, snap)) return;
      const int64_t nN = (int64_t)(snap[0] - base_f);
      base_f = snap[0];
      s++;
      if (leader) ctl->subrounds++;
      if (nN == 0) break;
      { int2 *t = F; F = N; N = t; }
      nCur = nN > a.item_cap ? a.item_cap : nN;
      if (nN > a.item_cap && leader) atomicExch(&ctl->err, TRUSS_ECHECK);
    }
    if (leader) {
      ctl->levels++;
      ctl->kmax = k;
    }
    k++;
  }
  // totals (one atomic per warp)
  for (int o = 16; o >= 1; o >>= 1) {
    n_entries += __shfl_down_sync(TR_FULL, n_entries, o);
    n_dec += __shfl_down_sync(TR_FULL, n_dec, o);
    n_scan += __shfl_down_sync(TR_FULL, n_scan, o);
  }
  if (lane == 0) {
    atomicAdd(&ctl->entries, n_entries);
    atomicAdd(&ctl->decrements, n_dec);
    atomicAdd(&ctl->scanned, n_scan);
  }
}

__global__ void k_peel_init(int64_t m, const int32_t *sup, int32_t *res, int32_t *stamp,
                            int32_t *alive, PeelCtl *ctl) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    res[e] = sup[e];
    stamp[e] = 0;
    alive[e] = (int32_t)e;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->minres[0] = INT_MAX;
    ctl->minres[1] = INT_MAX;
    ctl->minres[2] = INT_MAX;
  }
}

}  // namespace

int run_peel(Arena &A, const Csr &g, const SupportOut &so, const int2 *pairs, const PeelCfg &cfg,
             int32_t *truss, PeelResult *out, cudaStream_t s) {
  const int64_t m = g.m;
  *out = PeelResult{};
  if (m == 0) return TRUSS_OK;
  // items of one sub-round <= sum over its edges of max(1, ceil(sup / kItem))
  const int64_t item_cap = m + so.entries / kItem + 64;
  int32_t *res = A.get<int32_t>(m), *stamp = A.get<int32_t>(m);
  int32_t *al0 = A.get<int32_t>(m), *al1 = A.get<int32_t>(m);
  int2 *Q0 = A.get<int2>(item_cap), *Q1 = A.get<int2>(item_cap);
  PeelCtl *ctl = A.get<PeelCtl>(1);
  if (!res || !stamp || !al0 || !al1 || !Q0 || !Q1 || !ctl) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(ctl, 0, sizeof(PeelCtl), s));
  k_peel_init<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, so.sup, res, stamp, al0, ctl);
  TR_LAUNCHED();

  int dev = 0, sms = cfg.sms;
  TR_CUDA(cudaGetDevice(&dev));
  if (sms <= 0) TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int occ = 0;
  TR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_peel, kPeelBlock, 0));
  if (occ < 1) return TRUSS_ECUDA;
  if (cfg.blocks_per_sm > 0 && cfg.blocks_per_sm < occ) occ = cfg.blocks_per_sm;
  PeelArgs a{};
  a.m = m;
  a.toff = so.toff;
  a.sup = so.sup;
  a.pairs = pairs;
  a.res = res;
  a.stamp = stamp;
  a.truss = truss;
  a.alive0 = al0;
  a.alive1 = al1;
  a.Q0 = Q0;
  a.Q1 = Q1;
  a.item_cap = item_cap;
  a.ctl = ctl;
  a.wait_ns = cfg.wait_ns;
  const char *trace_path = getenv("TRUSS_TRACE");
  const int trace_cap = 1 << 20;
  if (trace_path) {
    a.trace = A.get<int4>(trace_cap);
    a.trace_cap = a.trace ? trace_cap : 0;
  }
  void *args[] = {&a};
  TR_CUDA(cudaLaunchCooperativeKernel((const void *)k_peel, dim3(sms * occ), dim3(kPeelBlock),
                                      args, 0, s));
  count_launches(1);
  PeelCtl h{};
  TR_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(PeelCtl), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  out->err = h.err;
  out->kmax = h.kmax;
  out->levels = h.levels;
  out->subrounds = h.subrounds;
  out->entries = h.entries;
  out->decrements = h.decrements;
  out->scanned = h.scanned;
  if (trace_path && a.trace) {
    const int nsub = h.subrounds < trace_cap ? h.subrounds : trace_cap;
    std::vector<int4> t((size_t)nsub);
    TR_CUDA(cudaMemcpy(t.data(), a.trace, sizeof(int4) * nsub, cudaMemcpyDeviceToHost));
    if (FILE *f = fopen(trace_path, "w")) {
      fprintf(f, "k,items\n");
      for (auto &x : t) fprintf(f, "%d,%d\n", x.x, x.y);
      fclose(f);
    }
  }
  if (h.err != 0) return h.err;
  return TRUSS_OK;
}

}  // namespace tr
