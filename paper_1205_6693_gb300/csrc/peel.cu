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
//  scan (per level k):  F = {alive e : res[e] <= k-2}; the minimum residual
//        of the other alive edges is taken, so an empty level jumps straight
//        to k = min res + 2.  The list of alive edges scanned is rewritten
//        without the removed ones once at least a quarter of it is dead.
//  sub-round:  for every e in F and every triangle {e, e1, e2} on e's list
//        whose edges are all still alive, the triangle is charged exactly
//        once, by the lowest-id edge among those of its edges that are in F:
//        that edge decrements the residual of each partner not in F.  A
//        partner whose residual crosses from k-1 to k-2 joins the next
//        frontier (warp-aggregated append).  F edges get truss number k.
//
// Load balance inside a sub-round (its time is that of the slowest warp):
// an edge that joins a frontier is staged by the warp that pushed it and
// expanded, when that warp flushes, into work items of kItem list entries
// each (at least one item, which also records its truss number); an
// item carries its edge, its entry count and the offset of its entries, so a
// warp goes from the item straight to the list.  Every warp takes 4 items per
// iteration, 8 lanes per item and 2 entries per lane (independent loads in
// flight).  A warp's share of a sub-round is then at most
// ceil(items / (4 * warps)) iterations, whatever the lengths of the lists.
// Appends are staged per warp in shared memory and flushed with one atomic
// reservation per buffer (the list lengths and offsets of a buffer's pushed
// edges are loaded together at the flush), and per-level reductions (minimum residual, alive
// count) are combined per block first: a single global counter hit by every
// warp would serialise the whole grid on one L2 address.
// Every scan and every sub-round is one phase, ended by one grid barrier.
// Appends of phase p reserve space through counter slot p % 3 (frontier
// items qf, alive-list entries qa), which is read after the barrier that
// ends p.  The leader zeroes slot (p+1) % 3 during phase p: that slot was
// last read at the start of phase p-1, and every block has passed the
// barrier ending p-1 before the leader can be in phase p.  A block that
// leaves a barrier early therefore never appends to a counter that a slow
// block has still to read.
//
// Edge state is one 16-bit tag per edge, stamp[e]: 0 = alive, tag(s) = in
// the frontier of sub-round s, any other value = removed earlier.  A partner
// pushed during sub-round s is tagged tag(s+1), which reads as alive during
// s, so one grid barrier per sub-round suffices.  Tags repeat every 65,534
// sub-rounds, so at least every 32,768 sub-rounds one extra grid-wide pass
// rewrites every tag but the current frontier's to kDead.  (A 2-byte stamp
// leaves more of L2 to the residuals, which are read at random.)  res[e] of
// a frontier edge is never touched during its sub-round and equals the
// number of its still-alive triangles, so a frontier edge with res 0 skips
// its list.
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
constexpr int kWarps = kPeelBlock / 32;
constexpr int kItem = 16;  // list entries per work item (8 lanes x 2)
constexpr int kWP = 32;    // pushed edges staged per warp (one per lane)
constexpr int kWA = 128;   // alive-list entries staged per warp

struct PeelCtl {
  unsigned long long bar;    // barrier arrivals so far (never reset)
  int err;
  int pad0;
  unsigned long long qf[3];  // frontier items appended in phase p (slot p % 3)
  unsigned long long qa[3];  // alive-list entries appended in phase p
  int minres[3];             // per scan (slot = scan index % 3)
  int live[3];               // alive edges left after each scan
  int levels, subrounds, kmax, ntrace;
  unsigned long long entries, decrements, scanned;
  unsigned long long dead, dead_earlier;  // counting runs
};

struct PeelArgs {
  int64_t m;
  const int32_t *sup;
  // list of e: own[own_off[e] ..] (own_cnt[e] entries), then rest[off[e] ..]
  const int2 *own;
  const int64_t *own_off;
  const int32_t *own_cnt;  // null: no own parts
  const int2 *rest;
  const int64_t *off;
  int32_t *res;
  uint16_t *stamp;
  int retag;  // sub-rounds between tag rewrites (1 .. kRetagMax)
  int32_t *truss;
  int32_t *alive0, *alive1;
  int4 *Q0, *Q1;      // frontier work items (make_item)
  int64_t item_cap;   // capacity of Q0 and Q1
  int4 *trace;        // optional: per phase (k, items or -1 for a scan, globaltimer lo/hi)
  int trace_cap;
  PeelCtl *ctl;
  long long wait_ns;
  int k_stop;  // last level to run (0 = all)
  // counting runs (the COUNT kernel): removal sub-round of every edge, and
  // per level k < lvl_cap the entries read, those of destroyed triangles, and
  // those of triangles destroyed in an earlier level (lvl[3k .. 3k+2])
  int32_t *when;
  unsigned long long *lvl;
  int lvl_cap;
};

__device__ __forceinline__ void prefetch_l1(const void *p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ int items_of(int len) { return len > 0 ? (len + kItem - 1) / kItem : 1; }

constexpr int kTagMod = 65534;
constexpr int kRetagMax = 32768;
constexpr uint16_t kDead = 0xFFFF;
// Tag of sub-round s >= 1: 1 .. kTagMod.
__device__ __forceinline__ uint16_t tag_of(int s) { return (uint16_t)(1 + (s - 1) % kTagMod); }

// A work item covers up to kItem consecutive entries of one edge's list:
// na from its own part at offset oa, then nb from its rest part at ob.
// Offsets have 42 bits (x = edge, y = na | nb << 5 | first << 10 | the high
// 10 bits of oa << 11 | those of ob << 21, z / w = the low words of oa / ob).
constexpr int64_t kOffLimit = (int64_t)1 << 42;

__device__ __forceinline__ int4 make_item(int e, int na, int nb, bool first, int64_t oa,
                                          int64_t ob) {
  const uint32_t hi = (uint32_t)na | ((uint32_t)nb << 5) | ((uint32_t)first << 10) |
                      ((uint32_t)((uint64_t)oa >> 32) & 0x3FFu) << 11 |
                      ((uint32_t)((uint64_t)ob >> 32) & 0x3FFu) << 21;
  return make_int4(e, (int)hi, (int)(uint32_t)oa, (int)(uint32_t)ob);
}

// Per-warp staging buffers in shared memory (counts are warp-uniform).
struct WarpBuf {
  int32_t *push;  // edges pushed to the next frontier, not yet expanded
  int np;
  int32_t *alive;
  int na;
};

// Expand the staged pushed edges into work items and append them to queue Q
// with one reservation.  The list length and offsets of all staged edges
// are loaded together here, once per flush, instead of one dependent round
// trip per push inside the sub-round's loop.
template <bool OWN>
__device__ __forceinline__ void flush_push(const PeelArgs &a, WarpBuf &wb, int4 *Q,
                                           unsigned long long *qctr) {
  const int np = wb.np;
  if (np == 0) return;
  const int lane = lane_id();
  const bool v = lane < np;
  const int p = v ? wb.push[lane] : 0;
  const int L = v ? __ldg(&a.sup[p]) : 0;
  const int64_t lb = v ? __ldg(&a.off[p]) : 0;
  const int cA = (OWN && v) ? __ldg(&a.own_cnt[p]) : 0;
  const int64_t la = (OWN && v) ? __ldg(&a.own_off[p]) : 0;
  const int n = v ? items_of(L) : 0;
  const int P = warp_incl_scan(n);
  const int tot = __shfl_sync(TR_FULL, P, 31);
  unsigned long long b = 0;
  if (lane == 0) b = atomicAdd(qctr, (unsigned long long)tot);
  const long long base = (long long)__shfl_sync(TR_FULL, b, 0);
  for (int u0 = 0; u0 < tot; u0 += 32) {
    const int t = u0 + lane;
    const int o = warp_owner(P, t < tot ? t : tot - 1);
    const int po = __shfl_sync(TR_FULL, p, o);
    const int Po = __shfl_sync(TR_FULL, P, o);
    const int no = __shfl_sync(TR_FULL, n, o);
    const int Lo = __shfl_sync(TR_FULL, L, o);
    const int cAo = OWN ? __shfl_sync(TR_FULL, cA, o) : 0;
    const int64_t lao = OWN ? __shfl_sync(TR_FULL, la, o) : 0;
    const int64_t lbo = __shfl_sync(TR_FULL, lb, o);
    const long long idx = base + t;
    if (t < tot && idx < a.item_cap) {
      const int it = t - (Po - no);
      const int start = it * kItem;
      const int cnt = Lo > 0 ? min(kItem, Lo - start) : 0;
      const int na = min(max(cAo - start, 0), cnt);
      Q[idx] = make_item(po, na, cnt - na, it == 0, lao + start, lbo + max(start - cAo, 0));
    }
  }
  __syncwarp();
  wb.np = 0;
}

__device__ __forceinline__ void flush_alive(const PeelArgs &a, WarpBuf &wb, int32_t *A2,
                                            unsigned long long *actr) {
  if (wb.na == 0) return;
  const int lane = lane_id();
  unsigned long long b = 0;
  if (lane == 0) b = atomicAdd(actr, (unsigned long long)wb.na);
  const long long b0 = (long long)__shfl_sync(TR_FULL, b, 0);
  for (int t = lane; t < wb.na; t += 32)
    if (b0 + t < a.m) A2[b0 + t] = wb.alive[t];
  __syncwarp();
  wb.na = 0;
}

// Queue the alive edges of the lanes with `keep` for the rewritten list.
__device__ __forceinline__ void push_alive(const PeelArgs &a, bool keep, int e, WarpBuf &wb,
                                           int32_t *A2, unsigned long long *actr) {
  const unsigned mask = __ballot_sync(TR_FULL, keep);
  if (mask == 0) return;
  const int tot = __popc(mask);
  if (wb.na + tot > kWA) flush_alive(a, wb, A2, actr);
  if (keep) wb.alive[wb.na + __popc(mask & ((1u << lane_id()) - 1u))] = e;
  __syncwarp();
  wb.na += tot;
}

// Push edge p (for each lane with `push`) to the next frontier: stamp it
// with tag `tagv` and stage it for expansion into work items.  All lanes
// call it.
template <bool OWN>
__device__ __forceinline__ void push_items(const PeelArgs &a, bool push, int p, WarpBuf &wb,
                                           int4 *Q, unsigned long long *qctr, uint16_t tagv) {
  const unsigned mask = __ballot_sync(TR_FULL, push);
  if (mask == 0) return;
  const int tot = __popc(mask);
  if (wb.np + tot > kWP) flush_push<OWN>(a, wb, Q, qctr);
  if (push) {
    a.stamp[p] = tagv;
    wb.push[wb.np + __popc(mask & ((1u << lane_id()) - 1u))] = p;
    // the flush reads p's list length and offsets: start fetching them now
    prefetch_l1(a.sup + p);
    prefetch_l1(a.off + p);
    if (OWN) {
      prefetch_l1(a.own_cnt + p);
      prefetch_l1(a.own_off + p);
    }
  }
  __syncwarp();
  wb.np += tot;
}

// Decide whether frontier edge e charges the triangle {e, p1, p2} in
// sub-round s: all three edges alive, and e the lowest-id frontier edge among
// them.  d1 / d2 = decrement p1 / p2 (the partners not in the frontier).
// ts / tn = tag(s) / tag(s+1).
__device__ __forceinline__ void decide(const PeelArgs &a, bool valid, int e, int2 pr, int ts,
                                       int tn, bool &d1, bool &d2, bool &dead) {
  d1 = d2 = dead = false;
  if (!valid) return;
  const int p1 = pr.x, p2 = pr.y;
  if ((uint32_t)p1 >= (uint32_t)a.m || (uint32_t)p2 >= (uint32_t)a.m) {
    atomicExch(&a.ctl->err, TRUSS_ECHECK);  // corrupt list entry: skip it
    return;
  }
  // more than half the entries read belong to triangles that already lost
  // an edge: partner 2's state is read only if partner 1 is still there
  const int s1 = __ldcg(&a.stamp[p1]);
  if (s1 != 0 && s1 != ts && s1 != tn) {
    dead = true;
    return;
  }
  const int s2 = __ldcg(&a.stamp[p2]);
  const bool dead1 = s1 != 0 && s1 != ts && s1 != tn, dead2 = s2 != 0 && s2 != ts && s2 != tn;
  dead = dead1 || dead2;
  if (dead) return;
  const bool in1 = s1 == ts, in2 = s2 == ts;
  if (!in1 && !in2) {
    d1 = true;
    d2 = true;
  } else if (in1 && !in2) {
    d2 = e < p1;  // e and e1 in F: the lower id charges e2
  } else if (!in1 && in2) {
    d1 = e < p2;
  }
}

// NE triangle entries per lane (all lanes call it; `v[i]` masks idle
// entries, e[i] is the frontier edge of entry i).  Each charged triangle
// decrements its partners outside the frontier; a partner whose residual
// crosses k-1 -> k-2 joins the next frontier.  All loads and atomics of the
// NE entries are issued before any result is used.
template <int NE, bool OWN, bool COUNT>
__device__ __forceinline__ void charge(const PeelArgs &a, const int *e, const bool *v,
                                       const int2 *p, int k, int ts, int tn, WarpBuf &wb,
                                       int4 *N, unsigned long long *qctr,
                                       unsigned &n_dec, int s_lvl0, unsigned &n_dead,
                                       unsigned &n_early) {
  bool d1[NE], d2[NE], dd[NE];
#pragma unroll
  for (int i = 0; i < NE; i++) decide(a, v[i], e[i], p[i], ts, tn, d1[i], d2[i], dd[i]);
  if (COUNT) {
    // a destroyed triangle lost its first edge when the earlier-removed of
    // its removed partners went (partners still alive have no removal yet)
#pragma unroll
    for (int i = 0; i < NE; i++) {
      if (!dd[i]) continue;
      const int w1 = __ldcg(&a.when[p[i].x]), w2 = __ldcg(&a.when[p[i].y]);
      n_dead++;
      n_early += min(w1, w2) < s_lvl0;
    }
  }
  int o1[NE], o2[NE];
#pragma unroll
  for (int i = 0; i < NE; i++) {
    o1[i] = d1[i] ? atomicSub(&a.res[p[i].x], 1) : INT_MAX;
    o2[i] = d2[i] ? atomicSub(&a.res[p[i].y], 1) : INT_MAX;
    n_dec += (unsigned)(d1[i] + d2[i]);
  }
  // pending pushes of this lane, bit 2i (p[i].x) and 2i+1 (p[i].y); the
  // warp pushes one per lane per step through a single push_items site
  unsigned pend = 0;
#pragma unroll
  for (int i = 0; i < NE; i++)
    pend |= (o1[i] == k - 1 ? 1u : 0u) << (2 * i) | (o2[i] == k - 1 ? 1u : 0u) << (2 * i + 1);
  while (__any_sync(TR_FULL, pend != 0)) {
    int q = 0;
    const bool has = pend != 0;
    if (has) {
      const int b = __ffs(pend) - 1;
      pend &= pend - 1;
#pragma unroll
      for (int i = 0; i < NE; i++)
        if ((b >> 1) == i) q = (b & 1) ? p[i].y : p[i].x;
    }
    push_items<OWN>(a, has, q, wb, N, qctr, (uint16_t)tn);
  }
}

// MINB = resident blocks per SM the register budget is sized for (1: up to
// 128 registers per thread, 2: 64); G = work items per 8-lane group per
// iteration (2 entries per lane per item).
// OWN: the lists keep own parts in the records (TriLists::own_cnt set).
template <int MINB, int G, bool OWN, bool COUNT = false>
__global__ void __launch_bounds__(kPeelBlock, MINB) k_peel(PeelArgs a) {
  const int lane = lane_id();
  const int wib = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * kWarps + wib;  // grids are one or two blocks per SM
  const int twarps = gridDim.x * kWarps;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  PeelCtl *ctl = a.ctl;
  __shared__ int32_t s_push[kWarps][kWP];
  __shared__ int32_t s_alive[kWarps][kWA];
  __shared__ int s_minres, s_live;
  WarpBuf wb{s_push[wib], 0, s_alive[wib], 0};
  if (threadIdx.x == 0) {
    s_minres = INT_MAX;
    s_live = 0;
  }
  __syncthreads();

  int k = 2, s = 1, sc = 0;
  unsigned ph = 0;  // phase index (scans and sub-rounds)
  int32_t *alive = a.alive0, *alive2 = a.alive1;
  int4 *F = a.Q0, *N = a.Q1;
  int64_t nAlive = a.m;
  bool compact = false;  // rewrite the alive list during this scan
  // per-lane work counts (32-bit: a lane's share of even 2^33 list entries
  // over the grid's 150 K lanes stays far below 2^32)
  unsigned n_entries = 0, n_dec = 0, n_scan = 0;
  unsigned n_dead = 0, n_early = 0;  // counting runs: totals so far
  // this warp's first work items of the coming sub-round, loaded right after
  // the barrier together with the item count instead of after it
  int4 pre[G];
  const int64_t it0 = (int64_t)gwarp * 4 * G + (lane >> 3);
  auto prefetch = [&](const int4 *Q) {
#pragma unroll
    for (int g = 0; g < G; g++)
      pre[g] = it0 + g * 4 < a.item_cap ? __ldcg(&Q[it0 + g * 4]) : make_int4(0, 0, 0, 0);
  };
  // Every a.retag sub-rounds (checked at the start of each phase, the same in
  // every block): tags other than the current frontier's become kDead.  A
  // tag left on a removed edge is then from the last a.retag sub-rounds, so
  // it never equals tag(s) or tag(s+1) of a later sub-round by wrapping.
  int last_retag = 0;
  auto retag = [&]() -> bool {
    if (s - last_retag < a.retag) return true;
    last_retag = s;
    const uint16_t keep = tag_of(s);
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.m; e += nt) {
      const uint16_t t = __ldcg(&a.stamp[e]);
      if (t != 0 && t != keep) a.stamp[e] = kDead;
    }
    return grid_barrier(&ctl->bar, &ctl->err, a.wait_ns);
  };

  for (;;) {
    if (a.k_stop > 0 && k > a.k_stop) break;  // k is the same in every block
    if (!retag()) return;
    // ------------------------------------------------------------ scan ---
    if (leader && a.trace && ctl->ntrace < a.trace_cap) {
      const unsigned long long t = global_ns();
      a.trace[ctl->ntrace++] = make_int4(k, -1, (int)(uint32_t)t, (int)(uint32_t)(t >> 32));
    }
    const int slot = sc % 3;
    unsigned long long *qf = &ctl->qf[ph % 3], *qa = &ctl->qa[ph % 3];
    if (leader) {
      ctl->minres[(sc + 1) % 3] = INT_MAX;
      ctl->live[(sc + 1) % 3] = 0;
      ctl->qf[(ph + 1) % 3] = 0;
      ctl->qa[(ph + 1) % 3] = 0;
    }
    int wmin = INT_MAX, wlive = 0;
    // 4 x 32 entries per warp iteration: all loads are issued before any
    // decision, so one dependent round trip covers 4 entries per lane
    constexpr int kScanU = 4;
    for (int64_t base = (int64_t)gwarp * 32 * kScanU; base < nAlive;
         base += (int64_t)twarps * 32 * kScanU) {
      int e[kScanU], st[kScanU], r[kScanU];
#pragma unroll
      for (int u = 0; u < kScanU; u++) {
        const int64_t i = base + u * 32 + lane;
        e[u] = i < nAlive ? __ldcg(&alive[i]) : -1;
      }
#pragma unroll
      for (int u = 0; u < kScanU; u++) {
        st[u] = e[u] >= 0 ? __ldcg(&a.stamp[e[u]]) : 1;
        r[u] = e[u] >= 0 ? __ldcg(&a.res[e[u]]) : 0;
      }
      unsigned pend = 0;  // entries of this lane that join the frontier
#pragma unroll
      for (int u = 0; u < kScanU; u++) {
        const bool live = e[u] >= 0 && st[u] == 0;
        const bool toF = live && r[u] <= k - 2;
        const bool keep = live && !toF;
        pend |= (toF ? 1u : 0u) << u;
        if (compact) push_alive(a, keep, e[u], wb, alive2, qa);
        wmin = min(wmin, __reduce_min_sync(TR_FULL, keep ? r[u] : INT_MAX));
        wlive += __popc(__ballot_sync(TR_FULL, keep));
        n_scan += (e[u] >= 0);
      }
      while (__any_sync(TR_FULL, pend != 0)) {
        int q = 0;
        const bool has = pend != 0;
        if (has) {
          const int b = __ffs(pend) - 1;
          pend &= pend - 1;
#pragma unroll
          for (int u = 0; u < kScanU; u++)
            if (b == u) q = e[u];
        }
        push_items<OWN>(a, has, q, wb, F, qf, tag_of(s));
      }
    }
    flush_push<OWN>(a, wb, F, qf);
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
    prefetch(F);
    const int minres = __ldcg(&ctl->minres[slot]);
    const int64_t live = __ldcg(&ctl->live[slot]);
    const int64_t nF = (int64_t)__ldcg(qf);
    if (compact) {
      nAlive = (int64_t)__ldcg(qa);
      int32_t *t = alive;
      alive = alive2;
      alive2 = t;
    }
    compact = 4 * live <= 3 * nAlive;  // rewrite the list once a quarter of it is dead
    sc++;
    if (nF == 0) {
      if (live == 0) break;
      k = minres + 2;  // every alive edge has res >= k-1: skip empty levels
      continue;
    }
    // --------------------------------------------------------- sub-rounds ---
    int64_t nCur = nF;
    const int s_lvl0 = s;  // first sub-round of this level
    for (;;) {
      const unsigned c_ent = n_entries, c_dead = n_dead, c_early = n_early;
      if (!retag()) return;
      const int ts = tag_of(s), tn = tag_of(s + 1);
      if (leader && a.trace && ctl->ntrace < a.trace_cap) {
        const unsigned long long t = global_ns();
        a.trace[ctl->ntrace++] = make_int4(k, (int)min(nCur, (int64_t)INT_MAX),
                                           (int)(uint32_t)t, (int)(uint32_t)(t >> 32));
      }
      unsigned long long *qn = &ctl->qf[ph % 3];
      if (leader) {
        ctl->qf[(ph + 1) % 3] = 0;
        ctl->qa[(ph + 1) % 3] = 0;
      }
      const int grp = lane >> 3, j = lane & 7;
      const int64_t stride = (int64_t)twarps * 4 * G;
      for (int64_t base = (int64_t)gwarp * 4 * G; base < nCur; base += stride) {
        // this iteration's items were loaded one iteration ahead (the first
        // right after the barrier); load the next iteration's now
        int4 cur[G];
#pragma unroll
        for (int g = 0; g < G; g++) {
          cur[g] = pre[g];
          const int64_t nx = base + stride + g * 4 + grp;
          pre[g] = nx < nCur ? __ldcg(&F[nx]) : make_int4(0, 0, 0, 0);
        }
        int ee[2 * G];
        bool vv[2 * G];
        int2 pp[2 * G];
        int na[G], cnt[G];
        int64_t la[G], lb[G];
#pragma unroll
        for (int g = 0; g < G; g++) {
          const int64_t it = base + g * 4 + grp;
          ee[2 * g] = 0;
          na[g] = 0;
          cnt[g] = 0;
          la[g] = 0;
          lb[g] = 0;
          if (it < nCur) {
            const int4 item = cur[g];
            const uint32_t hi = (uint32_t)item.y;
            ee[2 * g] = item.x;
            na[g] = OWN ? (int)(hi & 31u) : 0;
            cnt[g] = na[g] + ((hi >> 5) & 31u);
            la[g] = OWN ? (int64_t)(((uint64_t)((hi >> 11) & 0x3FFu) << 32) | (uint32_t)item.z) : 0;
            lb[g] = (int64_t)(((uint64_t)(hi >> 21) << 32) | (uint32_t)item.w);
            if (((hi >> 10) & 1u) && j == 0) {
              a.truss[item.x] = k;
              if (COUNT) a.when[item.x] = s;
            }
          }
          ee[2 * g + 1] = ee[2 * g];
        }
        int r[G];
#pragma unroll
        for (int g = 0; g < G; g++) {
          const bool ha = j < cnt[g], hb = j + 8 < cnt[g];
          r[g] = ha ? __ldcg(&a.res[ee[2 * g]]) : 0;
          // list entries are read once: evict-first, so that the residuals
          // and stamps (re-read at random) keep their place in L2
          const int2 *srcA = j < na[g] ? a.own + la[g] + j : a.rest + lb[g] + (j - na[g]);
          const int2 *srcB =
              j + 8 < na[g] ? a.own + la[g] + j + 8 : a.rest + lb[g] + (j + 8 - na[g]);
          pp[2 * g] = ha ? __ldcs(srcA) : make_int2(0, 0);
          pp[2 * g + 1] = hb ? __ldcs(srcB) : make_int2(0, 0);
          vv[2 * g] = ha;
          vv[2 * g + 1] = hb;
        }
#pragma unroll
        for (int g = 0; g < G; g++) {
          vv[2 * g] = vv[2 * g] && r[g] > 0;
          vv[2 * g + 1] = vv[2 * g + 1] && r[g] > 0;
          n_entries += (unsigned)(vv[2 * g] + vv[2 * g + 1]);
        }
        // the next iteration's items have arrived by now: start fetching
        // their list entries (into L1; the lists are read-only here) and
        // their edges' residuals (into L2) while this iteration charges
#pragma unroll
        for (int g = 0; g < G; g++) {
          const uint32_t hi = (uint32_t)pre[g].y;
          const int nna = OWN ? (int)(hi & 31u) : 0;
          const int ncnt = nna + (int)((hi >> 5) & 31u);
          const int64_t nla =
              OWN ? (int64_t)(((uint64_t)((hi >> 11) & 0x3FFu) << 32) | (uint32_t)pre[g].z) : 0;
          const int64_t nlb = (int64_t)(((uint64_t)(hi >> 21) << 32) | (uint32_t)pre[g].w);
          if (j < ncnt) prefetch_l1(j < nna ? a.own + nla + j : a.rest + nlb + (j - nna));
          if (j + 8 < ncnt)
            prefetch_l1(j + 8 < nna ? a.own + nla + j + 8 : a.rest + nlb + (j + 8 - nna));
          if (j == 0 && ncnt > 0) prefetch_l2(a.res + pre[g].x);
        }
        charge<2 * G, OWN, COUNT>(a, ee, vv, pp, k, ts, tn, wb, N, qn, n_dec, s_lvl0, n_dead,
                                  n_early);
      }
      flush_push<OWN>(a, wb, N, qn);
      if (COUNT && k < a.lvl_cap) {
        unsigned x0 = n_entries - c_ent, x1 = n_dead - c_dead, x2 = n_early - c_early;
        for (int o = 16; o >= 1; o >>= 1) {
          x0 += __shfl_down_sync(TR_FULL, x0, o);
          x1 += __shfl_down_sync(TR_FULL, x1, o);
          x2 += __shfl_down_sync(TR_FULL, x2, o);
        }
        if (lane == 0 && (x0 | x1 | x2)) {
          atomicAdd(&a.lvl[3 * k], (unsigned long long)x0);
          atomicAdd(&a.lvl[3 * k + 1], (unsigned long long)x1);
          atomicAdd(&a.lvl[3 * k + 2], (unsigned long long)x2);
        }
      }
      if (!grid_barrier(&ctl->bar, &ctl->err, a.wait_ns)) return;
      ph++;
      prefetch(N);
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
  if (leader && a.trace && ctl->ntrace < a.trace_cap) {
    const unsigned long long t = global_ns();
    a.trace[ctl->ntrace++] = make_int4(k, -2, (int)(uint32_t)t, (int)(uint32_t)(t >> 32));
  }
  // totals (one atomic per warp)
  for (int o = 16; o >= 1; o >>= 1) {
    n_entries += __shfl_down_sync(TR_FULL, n_entries, o);
    n_dec += __shfl_down_sync(TR_FULL, n_dec, o);
    n_scan += __shfl_down_sync(TR_FULL, n_scan, o);
    if (COUNT) {
      n_dead += __shfl_down_sync(TR_FULL, n_dead, o);
      n_early += __shfl_down_sync(TR_FULL, n_early, o);
    }
  }
  if (lane == 0) {
    atomicAdd(&ctl->entries, (unsigned long long)n_entries);
    atomicAdd(&ctl->decrements, (unsigned long long)n_dec);
    atomicAdd(&ctl->scanned, (unsigned long long)n_scan);
    if (COUNT) {
      atomicAdd(&ctl->dead, (unsigned long long)n_dead);
      atomicAdd(&ctl->dead_earlier, (unsigned long long)n_early);
    }
  }
}

// Residual given to pinned edges: no level ever reaches it, and the
// decrements it can receive (at most its support) leave it out of reach.
constexpr int kPinnedRes = INT_MAX / 4;

__global__ void k_peel_init(int64_t m, const int32_t *sup, const uint8_t *pinned, int32_t *res,
                            uint16_t *stamp, int32_t *alive, int32_t *truss, PeelCtl *ctl) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    res[e] = (pinned && pinned[e]) ? kPinnedRes : sup[e];
    stamp[e] = 0;
    alive[e] = (int32_t)e;
    truss[e] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = 0; i < 3; i++) {
      ctl->minres[i] = INT_MAX;
      ctl->live[i] = 0;
    }
  }
}

// Removal-order figures of a counting run (PeelResult): min alive degrees
// from the removal sub-rounds, the edges present at each level that removes
// one (from the truss-number histogram), and the per-level entry counts,
// written to the file named by TRUSS_LEVEL_STATS if set.
__global__ void k_truss_hist(int64_t m, const int32_t *truss, int cap,
                             unsigned long long *cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = truss[e];
    if (k >= 0 && k < cap) atomicAdd(&cnt[k], 1ull);
  }
}

int count_run(Arena &A, const Csr &g, const SupportOut &so, const PeelArgs &a, const PeelCtl &h,
              const int32_t *truss, PeelResult *out, cudaStream_t s) {
  const int cap = h.kmax + 2 < a.lvl_cap ? h.kmax + 2 : a.lvl_cap;
  unsigned long long *cnt = A.get<unsigned long long>(cap);
  if (!cnt) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * cap, s));
  k_truss_hist<<<grid_for(g.m, 256, 152 * 16), 256, 0, s>>>(g.m, truss, cap, cnt);
  TR_LAUNCHED();
  std::vector<unsigned long long> hc((size_t)cap), hl((size_t)3 * cap);
  TR_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(unsigned long long) * cap,
                          cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaMemcpyAsync(hl.data(), a.lvl, sizeof(unsigned long long) * 3 * cap,
                          cudaMemcpyDeviceToHost, s));
  unsigned long long sums[2] = {0, 0};
  TR_TRY(count_min_alive(A, g, so, a.when, sums, s));
  TR_CUDA(cudaStreamSynchronize(s));
  // edges present when level k starts: truss number >= k
  std::vector<unsigned long long> alive((size_t)cap + 1, 0);
  for (int k = cap - 1; k >= 0; k--) alive[k] = alive[k + 1] + hc[k];
  out->alive_levels = 0;
  for (int k = 0; k < cap; k++)
    if (hc[k] > 0) out->alive_levels += alive[k];
  out->sum_min_alive = sums[0];
  out->sum_min_alive_start = sums[1];
  out->dead = h.dead;
  out->dead_earlier = h.dead_earlier;
  if (const char *path = getenv("TRUSS_LEVEL_STATS")) {
    if (FILE *f = fopen(path, "w")) {
      fprintf(f, "k,removed,present,entries,dead,dead_earlier\n");
      for (int k = 0; k < cap; k++)
        if (hc[k] > 0 || hl[3 * k] > 0)
          fprintf(f, "%d,%llu,%llu,%llu,%llu,%llu\n", k, hc[k], alive[k], hl[3 * k],
                  hl[3 * k + 1], hl[3 * k + 2]);
      fclose(f);
    }
  }
  return TRUSS_OK;
}

// Keys (endpoint, removal sub-round) of both endpoints of every edge.
__global__ void k_when_keys(int64_t m, const int32_t *esrc, const int32_t *adjp,
                            const int32_t *when, uint64_t *keys) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t w = (uint32_t)when[e];
    keys[2 * e] = (uint64_t)(uint32_t)esrc[e] << 32 | w;
    keys[2 * e + 1] = (uint64_t)(uint32_t)adjp[e] << 32 | w;
  }
}

// Degree of every vertex (out-edges + in-edges); entry n is 0.
__global__ void k_sym_degree(int64_t n, const int64_t *offp, const int64_t *inoff,
                             int64_t *deg) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u <= n;
       u += (int64_t)gridDim.x * blockDim.x)
    deg[u] = u < n ? (offp[u + 1] - offp[u]) + (inoff[u + 1] - inoff[u]) : 0;
}

// Entries of the sorted run keys[lo, hi) that are >= key.
__device__ __forceinline__ int64_t count_ge(const uint64_t *keys, int64_t lo, int64_t hi,
                                            uint64_t key) {
  const int64_t end = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (keys[mid] < key) lo = mid + 1; else hi = mid;
  }
  return end - lo;
}

// acc[0] += min over e's endpoints x of (1 + x's edges removed in a later
// sub-round than e); acc[1] += the same with every edge not removed before
// e's sub-round (e's co-frontier edges included).
__global__ void k_min_alive(int64_t m, const int32_t *esrc, const int32_t *adjp,
                            const int32_t *when, const int64_t *soff, const uint64_t *keys,
                            unsigned long long *acc) {
  unsigned long long lo = 0, hi = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int u = esrc[e], v = adjp[e];
    const uint64_t w = (uint32_t)when[e];
    const uint64_t ku = (uint64_t)(uint32_t)u << 32 | w, kv = (uint64_t)(uint32_t)v << 32 | w;
    const int64_t su = count_ge(keys, soff[u], soff[u + 1], ku);
    const int64_t sv = count_ge(keys, soff[v], soff[v + 1], kv);
    const int64_t au = 1 + count_ge(keys, soff[u], soff[u + 1], ku + 1);
    const int64_t av = 1 + count_ge(keys, soff[v], soff[v + 1], kv + 1);
    hi += (unsigned long long)(su < sv ? su : sv);
    lo += (unsigned long long)(au < av ? au : av);
  }
  for (int o = 16; o >= 1; o >>= 1) {
    lo += __shfl_down_sync(TR_FULL, lo, o);
    hi += __shfl_down_sync(TR_FULL, hi, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (lo) atomicAdd(&acc[0], lo);
    if (hi) atomicAdd(&acc[1], hi);
  }
}

}  // namespace

int count_min_alive(Arena &A, const Csr &g, const SupportOut &so, const int32_t *when,
                    unsigned long long *sum, cudaStream_t s) {
  const int64_t m = g.m, n = g.n;
  sum[0] = sum[1] = 0;
  if (m == 0) return TRUSS_OK;
  if (!so.inoff) return TRUSS_EINVAL;
  uint64_t *k0 = A.get<uint64_t>(2 * m), *k1 = A.get<uint64_t>(2 * m);
  int64_t *deg = A.get<int64_t>(n + 1), *soff = A.get<int64_t>(n + 1);
  unsigned long long *acc = A.get<unsigned long long>(2);
  if (!k0 || !k1 || !deg || !soff || !acc) return TRUSS_ENOMEM;
  k_when_keys<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, g.esrc, g.adjp, when, k0);
  TR_LAUNCHED();
  k_sym_degree<<<grid_for(n + 1, 256, 152 * 16), 256, 0, s>>>(n, g.offp, so.inoff, deg);
  TR_LAUNCHED();
  const int end_bit = 32 + bits_for((uint64_t)(n > 0 ? n - 1 : 0));
  size_t tb = 0, tb2 = 0;
  TR_TRY(sort_keys_u64(nullptr, &tb, k0, k1, 2 * m, 0, end_bit, s));
  TR_TRY(exclusive_sum_i64(nullptr, &tb2, deg, soff, n + 1, s));
  void *tmp = A.alloc(tb > tb2 ? tb : tb2);
  if (!tmp) return TRUSS_ENOMEM;
  TR_TRY(sort_keys_u64(tmp, &tb, k0, k1, 2 * m, 0, end_bit, s));
  TR_TRY(exclusive_sum_i64(tmp, &tb2, deg, soff, n + 1, s));
  TR_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), s));
  k_min_alive<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, g.esrc, g.adjp, when, soff, k1, acc);
  TR_LAUNCHED();
  TR_CUDA(cudaMemcpyAsync(sum, acc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  return TRUSS_OK;
}

int run_peel(Arena &A, const Csr &g, const SupportOut &so, const TriLists &L, const PeelCfg &cfg,
             int32_t *truss, PeelResult *out, cudaStream_t s) {
  const int64_t m = g.m;
  *out = PeelResult{};
  if (m == 0) return TRUSS_OK;
  // item offsets carry 42 bits
  if (so.entries >= kOffLimit || (L.own_cnt && so.records >= kOffLimit)) return TRUSS_EINVAL;
  if (so.entries > 0 && (!L.rest || !L.off || (L.own_cnt && (!L.own || !L.own_off))))
    return TRUSS_EINVAL;
  // items of one sub-round <= sum over its edges of max(1, ceil(sup / kItem))
  const int64_t item_cap = m + so.entries / kItem + 64;
  int32_t *res = A.get<int32_t>(m);
  uint16_t *stamp = A.get<uint16_t>(m);
  int32_t *al0 = A.get<int32_t>(m), *al1 = A.get<int32_t>(m);
  int4 *Q0 = A.get<int4>(item_cap), *Q1 = A.get<int4>(item_cap);
  PeelCtl *ctl = A.get<PeelCtl>(1);
  if (!res || !stamp || !al0 || !al1 || !Q0 || !Q1 || !ctl) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(ctl, 0, sizeof(PeelCtl), s));
  k_peel_init<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, so.sup, cfg.pinned, res, stamp, al0,
                                                          truss, ctl);
  TR_LAUNCHED();

  int dev = 0, sms = cfg.sms;
  TR_CUDA(cudaGetDevice(&dev));
  if (sms <= 0) TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // variant 1: 128-register kernel taking 2 items per lane group, one block
  // per SM; 3: 1 item per group, one block per SM; otherwise (0, 2) the
  // 64-register kernel with 1 item per group and two blocks per SM
  const int variant = cfg.variant == 1 ? 1 : (cfg.variant == 3 ? 3 : 2);
  const bool own = L.own_cnt != nullptr;
  const void *kern;
  if (cfg.count) {
    kern = own ? (const void *)k_peel<2, 1, true, true> : (const void *)k_peel<2, 1, false, true>;
  } else if (own) {
    kern = variant == 1   ? (const void *)k_peel<1, 2, true>
           : variant == 3 ? (const void *)k_peel<1, 1, true>
                          : (const void *)k_peel<2, 1, true>;
  } else {
    kern = variant == 1   ? (const void *)k_peel<1, 2, false>
           : variant == 3 ? (const void *)k_peel<1, 1, false>
                          : (const void *)k_peel<2, 1, false>;
  }
  int occ = 0;
  TR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPeelBlock, 0));
  if (occ < 1) return TRUSS_ECUDA;
  if (variant != 2 && !cfg.count && occ > 1) occ = 1;
  PeelArgs a{};
  a.m = m;
  a.sup = so.sup;
  a.own = L.own;
  a.own_off = L.own_off;
  a.own_cnt = L.own_cnt;
  a.rest = L.rest;
  a.off = L.off ? L.off : so.toff;
  a.res = res;
  a.stamp = stamp;
  a.retag = kRetagMax;
  if (const char *rt = getenv("TRUSS_PEEL_RETAG")) {  // testing: rewrite tags more often
    const int v = atoi(rt);
    a.retag = v < 1 ? 1 : v > kRetagMax ? kRetagMax : v;
  }
  a.truss = truss;
  a.alive0 = al0;
  a.alive1 = al1;
  a.Q0 = Q0;
  a.Q1 = Q1;
  a.item_cap = item_cap;
  a.ctl = ctl;
  a.wait_ns = cfg.wait_ns;
  a.k_stop = cfg.k_stop;
  constexpr int kLvlCap = 1 << 16;
  if (cfg.count) {
    a.when = A.get<int32_t>(m);
    a.lvl = A.get<unsigned long long>(3 * (int64_t)kLvlCap);
    if (!a.when || !a.lvl) return TRUSS_ENOMEM;
    a.lvl_cap = kLvlCap;
    TR_CUDA(cudaMemsetAsync(a.when, 0x7F, sizeof(int32_t) * m, s));  // never removed
    TR_CUDA(cudaMemsetAsync(a.lvl, 0, sizeof(unsigned long long) * 3 * kLvlCap, s));
  }
  const char *trace_path = getenv("TRUSS_TRACE");
  const int trace_cap = 1 << 20;
  if (trace_path) {
    a.trace = A.get<int4>(trace_cap);
    a.trace_cap = a.trace ? trace_cap : 0;
  }
  void *args[] = {&a};
  TR_CUDA(cudaLaunchCooperativeKernel(kern, dim3(sms * occ), dim3(kPeelBlock), args, 0, s));
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
    const int nt = h.ntrace < trace_cap ? h.ntrace : trace_cap;
    std::vector<int4> t((size_t)nt);
    TR_CUDA(cudaMemcpy(t.data(), a.trace, sizeof(int4) * nt, cudaMemcpyDeviceToHost));
    if (FILE *f = fopen(trace_path, "w")) {
      fprintf(f, "k,items,t_ns\n");  // items: -1 = level scan, -2 = end
      for (auto &x : t)
        fprintf(f, "%d,%d,%llu\n", x.x, x.y,
                ((unsigned long long)(uint32_t)x.w << 32) | (uint32_t)x.z);
      fclose(f);
    }
  }
  if (h.err != 0) return h.err;
  if (cfg.count) TR_TRY(count_run(A, g, so, a, h, truss, out, s));
  return TRUSS_OK;
}

}  // namespace tr
