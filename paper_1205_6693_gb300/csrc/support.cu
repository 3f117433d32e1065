// Edge support (Definition 1; Algorithm 2 step 2) and per-edge triangle lists.
//
// Vertices are ranked by (degree, id) and every edge points from its
// lower-ranked end u to its higher-ranked end v (the degree order of
// Theorem 1).  A triangle u < v < w is found once, from its middle vertex v
// (k_support_v, below): w lies in out(v) and in out(u) after v.  Its edges
// are e_uv, e_uw (both in out(u)) and e_vw (in out(v)).  Counts: supA[e] =
// triangles in which e is e_uv or e_uw, supB[e] = triangles in which it is
// e_vw; sup = supA + supB.
//
// The walk also records each triangle as (e_uw, e_vw) in a region of e_uv
// (the triangle records), from which two streaming passes build the dense
// per-edge lists list(e) = pairs[toff[e] .. toff[e] + sup[e]).  When the
// records do not fit in device memory, a second, owner-by-owner walk
// (k_list_walk) writes the lists directly: for v in out(u) it intersects
// out(v) with the part of out(u) after v by a warp merge path (out(v) staged
// in chunks, the window of out(u) cut to the chunk's value range, the merged
// sequence split evenly over the 32 lanes), and writes one entry into each of
// the triangle's three lists.
#include <climits>

#include "engine.h"

namespace tr {

namespace {

constexpr int kBlock = 256;
constexpr int64_t kRangeWork = 16384;  // target walk cost per range
constexpr int kEdgeCost = 64;          // fixed walk cost per oriented edge (entries)
// Head walk (support): out(v) of up to kHeadCap entries staged per warp with
// its counts (int32) and a position table of kHashSlots uint16 slots.
constexpr int kHeadCap = 512;
// Out-lists shorter than this are not staged: their few probes go to the
// L1-cached global list (batch of small graphs: support 11.1 -> 10.3 ms).
constexpr int kStageMin = 16;
constexpr int kHashSlots = 2048;
constexpr size_t kHeadSmem = (size_t)kHeadCap * 8 + (size_t)kHashSlots * 2;
// List walk (the list builder used when the triangle records do not fit):
// out(u) of up to kListCap entries staged with its cursors (int64), and out(v)
// staged kAChunk entries at a time.
constexpr int kListCap = 256;
constexpr int kAChunk = 512;
constexpr size_t kListSmem = (size_t)kListCap * 12 + (size_t)kAChunk * 4;

// Arguments of the list walk (owner by owner, lists written directly).
struct ListArgs {
  int64_t n, m;
  const int64_t *offp;
  const int32_t *adjp;
  const int32_t *esrc;
  const int64_t *wpre;  // [m+1] exclusive prefix of the owner-centric walk cost
  const int64_t *rb;    // [P+1] range r = edges [rb[r], rb[r+1])
  int64_t W;            // total walk cost
  int64_t P;            // number of ranges
  int stage_max;        // stage out(u) in shared memory when |out(u)| <= this
  unsigned long long *curA;  // next slot of e's owner part (starts at toff[e])
  unsigned long long *curB;  // next slot of e's other part (toff[e] + supA[e])
  int2 *pairs;
  int64_t entries;      // size of pairs (writes beyond it are dropped)
  int *err;             // set to TRUSS_ECHECK if a list would overflow
};

// r W / P without overflowing 64 bits (r <= P <= m).
__device__ __forceinline__ int64_t range_point(int64_t W, int64_t P, int64_t r) {
  return (W / P) * r + (W % P) * r / P;
}

// First e in [0, m] with wpre[e] >= x.
__device__ __forceinline__ int64_t lower_bound64(const int64_t *a, int64_t m, int64_t x) {
  int64_t lo = 0, hi = m;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (__ldg(&a[mid]) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Out-list of u as seen by one warp: staged in shared memory (STAGED) or
// read from global memory.  A compile-time choice, so the staged case
// compiles to plain shared-memory loads.
template <bool STAGED>
struct OutList {
  const int32_t *L;
  int d;

  __device__ __forceinline__ int at(int i) const { return STAGED ? L[i] : __ldg(&L[i]); }

  // Lower bound of w in L[lo, d): a branch-free search whose step count
  // depends only on d - lo, which is the same for every lane of the warp.
  __device__ __forceinline__ int lower(int lo, int w) const {
    const int span = d - lo;
    int q = lo;
    if (span > 0) {
      for (int step = 1 << (31 - __clz(span)); step > 0; step >>= 1) {
        const int nq = q + step;
        if (nq <= d && at(nq - 1) < w) q = nq;
      }
    }
    return q;
  }
};

// Write the triangle (u, v, w), found as out(v)[evw - ob] == L[q] while
// walking edge (u, L[io]), into its three lists.  C = the owner cursors of
// out(u) (shared or global).
__device__ __forceinline__ void found(const ListArgs &a, int64_t bu, unsigned long long *C,
                                      int io, int q, int64_t evw) {
  const int64_t euv = bu + io, euw = bu + q;
  const int64_t x1 = (int64_t)atomicAdd(&C[io], 1ull);
  const int64_t x2 = (int64_t)atomicAdd(&C[q], 1ull);
  const int64_t x3 = (int64_t)atomicAdd(&a.curB[evw], 1ull);
  if (x1 < a.entries && x2 < a.entries && x3 < a.entries) {
    a.pairs[x1] = make_int2((int)euw, (int)evw);
    a.pairs[x2] = make_int2((int)euv, (int)evw);
    a.pairs[x3] = make_int2((int)euv, (int)euw);
  } else {
    atomicExch(a.err, TRUSS_ECHECK);
  }
}

// Walk edges (u, L[i]) for i in [i0, i1) (i1 <= d-1); bu = offp[u].
// For v = L[i], the triangles (u, v, w) are the common entries of out(v) and
// L[i+1, d).  out(v) is staged chunk by chunk in Abuf; the window of L is cut
// to [lower(chunk min), lower(chunk max + 1)) and the two sorted runs are
// intersected by a merge path: lane l takes positions [l*K, (l+1)*K) of the
// merged order (A first on ties), finds its start by a binary search on its
// diagonal and then merges K steps; an A entry equal to the current B head
// is a triangle.
template <bool STAGED>
__device__ __forceinline__ void walk(const ListArgs &a, int64_t bu, const OutList<STAGED> &ol,
                                     unsigned long long *C, int i0, int i1, int32_t *Abuf) {
  const int lane = lane_id();
  const int d = ol.d;
  const int Lmax = ol.at(d - 1);
  for (int c0 = i0; c0 < i1; c0 += 32) {
    const int i = c0 + lane;
    const bool valid = i < i1;
    const int v = valid ? ol.at(i) : 0;
    const int64_t vb = valid ? __ldg(&a.offp[v]) : 0;
    const int len = valid ? (int)(__ldg(&a.offp[v + 1]) - vb) : 0;
    const int nv = min(32, i1 - c0);
    for (int o = 0; o < nv; o++) {
      const int64_t ob = __shfl_sync(TR_FULL, vb, o);
      const int olen = __shfl_sync(TR_FULL, len, o);
      const int io = c0 + o;
      int blo = io + 1;
      for (int cA = 0; cA < olen && blo < d; cA += kAChunk) {
        const int ac = min(kAChunk, olen - cA);
        __syncwarp();
        for (int t = lane; t < ac; t += 32) Abuf[t] = __ldg(&a.adjp[ob + cA + t]);
        __syncwarp();
        const int amin = Abuf[0], amax = Abuf[ac - 1];
        if (amin > Lmax) break;  // nothing later in out(v) can be in out(u)
        blo = ol.lower(blo, amin);
        const int bhi = ol.lower(blo, amax + 1);
        const int bc = bhi - blo;
        if (bc > 0) {
          const int total = ac + bc;
          const int K = (total + 31) >> 5;
          int p = min(lane * K, total);
          const int pend = min(p + K, total);
          // merge-path split of diagonal p: A[0, ia) and B[0, p - ia) come first
          int lo = max(0, p - bc), hi = min(p, ac);
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (Abuf[mid] <= ol.at(blo + p - 1 - mid)) lo = mid + 1; else hi = mid;
          }
          int ia = lo, jb = p - lo;
          int av = ia < ac ? Abuf[ia] : INT_MAX;
          int bv = jb < bc ? ol.at(blo + jb) : INT_MAX;
          for (; p < pend; p++) {
            const bool takeA = av <= bv;
            if (takeA && av == bv) found(a, bu, C, io, blo + jb, ob + cA + ia);
            ia += takeA;
            jb += !takeA;
            av = ia < ac ? Abuf[ia] : INT_MAX;
            bv = jb < bc ? ol.at(blo + jb) : INT_MAX;
          }
        }
        blo = bhi;
      }
    }
  }
}

// Slot of vertex w in a position table of 2^(32 - sh) slots.
__device__ __forceinline__ unsigned hslot(int w, int sh) {
  return ((unsigned)w * 0x9E3779B1u) >> sh;
}

// ------------------------------------------------ head-centric support ---
// The support walk proper: every triangle (u, v, w) with rank u < v < w is
// found once, from its middle vertex v.  out(v) is staged in shared memory
// with a hash table of positions (out-lists of more than stage_max entries
// are searched in global memory instead), and for every in-edge (u, v) the
// entries of out(u) after v are looked up in it; a hit w at position q of
// out(v) is the triangle with e_uv = (u, v), e_uw = w's position in out(u)
// and e_vw = offp[v] + q.  Entries of out(u) after v are exactly the
// candidates (w must rank above v), so the work of an edge is |out(u) after
// v| rather than |out(v)|: sum over u of d(d-1)/2 for out-degrees d, which
// on power-law graphs is a few times smaller than the sum of |out(v)| over
// the edges (u, v).
// Counts: supA[e] = triangles in which e is e_uv or e_uw (both in out(u)),
// supB[e] = triangles in which it is e_vw; sup = supA + supB.
struct SupVArgs {
  int64_t n, m;
  const int64_t *offp;
  const int32_t *adjp;
  const int32_t *esrc;
  const int32_t *inedge;  // [m] edges grouped by head
  const int32_t *ihead;   // [m] head of inedge[i]
  const int64_t *inoff;   // [n+1] start of each head's group
  const int64_t *wcost;   // [m] walk cost of inedge[i]: |out(u) after v| + ecost
  const int64_t *wpre;    // [m+1] exclusive prefix of the walk cost, in inedge order
  const int64_t *rb;      // [P+1] range r = inedge positions [rb[r], rb[r+1])
  int64_t W, P;
  int ecost;      // the fixed part of wcost
  int stage_min;  // out-lists shorter than this are searched in global memory
  int stage_max;  // out-lists staged with their counts up to this many entries
  int hash_max;   // longer ones get a shared table of positions up to this many
  int32_t *supA, *supB;
  // optional: per edge e = (u, v), the triangles (u, v, w) it closes, as
  // (e_uw, e_vw) records in tb[tbpre[e] .. tbpre[e] + cuv[e])
  const int64_t *tbpre;  // [m+1] exclusive prefix of min(|out(v)|, |out(u) after v|)
  int2 *tb;
  int32_t *cuv;
};

// How a head's out(v) is searched: kSearch = branch-free search of the
// global list; kStaged = out(v) and its counts in shared memory with a hash
// table of positions; kHashOnly = a shared hash table of positions only
// (the warp's whole buffer), hits checked against the global list (L1) and
// counted with global atomics, for heads too long to stage.
constexpr int kSearch = 0, kStaged = 1, kHashOnly = 2;
constexpr int kHashOnlyCap = (int)(kHeadSmem / 2 / 2);  // heads up to this many entries

// Position of w in out(v) (kStaged: hash table Hs of size 2^(32-sh) over Ls;
// kHashOnly: the same over the global list gl), or -1.
template <int MODE>
__device__ __forceinline__ int find_in_out(int w, const int32_t *Ls, const unsigned short *Hs,
                                           int S, int sh, const int32_t *gl, int d) {
  if (MODE != kSearch) {
    unsigned sl = hslot(w, sh);
    for (;;) {
      const int p = Hs[sl];
      if (p == 0) return -1;
      if ((MODE == kStaged ? Ls[p - 1] : __ldg(&gl[p - 1])) == w) return p - 1;
      sl = (sl + 1) & (unsigned)(S - 1);
    }
  } else {
    int q = 0;
    for (int step = 1 << (31 - __clz(d)); step > 0; step >>= 1) {
      const int nq = q + step;
      if (nq <= d && __ldg(&gl[nq - 1]) < w) q = nq;
    }
    return (q < d && __ldg(&gl[q]) == w) ? q : -1;
  }
}

// Walks of at most kShortWalk entries are spread over the lanes, several
// edges per warp step; longer ones take the warp one edge at a time.
constexpr int kShortWalk = 128;
constexpr int kFlatU = 4;  // flattened steps whose loads are issued together

// One hit of the walk: triangle (u, v, w) with e_uw = euw and e_vw at
// position q of out(v), recorded at slot `slot` of e_uv's region.
template <int MODE>
__device__ __forceinline__ void count_hit(const SupVArgs &a, int32_t *Cs, int64_t bv, int q,
                                          int64_t euw, int64_t slot) {
  if (MODE == kStaged) atomicAdd(&Cs[q], 1);
  else atomicAdd(&a.supB[bv + q], 1);
  atomicAdd(&a.supA[euw], 1);
  if (a.tb) a.tb[slot] = make_int2((int)euw, (int)(bv + q));
}

// The in-edges inedge[i0 .. i1) of head v (bv = offp[v], dv = |out(v)|).
template <int MODE>
__device__ __forceinline__ void head_walk(const SupVArgs &a, int64_t i0, int64_t i1, int64_t bv,
                                          int dv, int vmax, const int32_t *Ls, int32_t *Cs,
                                          const unsigned short *Hs, int S, int sh) {
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t c0 = i0; c0 < i1; c0 += 32) {
    const int64_t j = c0 + lane;
    const bool valid = j < i1;
    // the walk length comes with the edge (its cost, by position), not from
    // the tail's offsets: two dependent loads fewer before the walk starts
    const int e = valid ? __ldg(&a.inedge[j]) : 0;
    const int len = valid ? (int)(__ldg(&a.wcost[j]) - a.ecost) : 0;  // out(u) after v
    const int64_t rb = (valid && a.tb) ? __ldg(&a.tbpre[e]) : 0;

    // short walks, flattened: step t of the warp is entry t - base(o) of
    // the walk of lane o = the owner of t (base = exclusive prefix of sl)
    const bool shrt = len <= kShortWalk;
    const int sl = shrt ? len : 0;
    const int P = warp_incl_scan(sl);
    const int total = __shfl_sync(TR_FULL, P, 31);
    int mycnt = 0;  // triangles found so far for this lane's (short) edge
    for (int t0 = 0; t0 < total; t0 += 32 * kFlatU) {
      int w[kFlatU], own[kFlatU], bo[kFlatU];
#pragma unroll
      for (int k = 0; k < kFlatU; k++) {
        const int t = t0 + k * 32 + lane;
        const bool act = t < total;
        own[k] = warp_owner(P, act ? t : total - 1);
        const int Po = __shfl_sync(TR_FULL, P, own[k]), so = __shfl_sync(TR_FULL, sl, own[k]);
        const int eo = __shfl_sync(TR_FULL, e, own[k]);
        bo[k] = Po - so;
        w[k] = act ? __ldg(&a.adjp[(int64_t)eo + 1 + (t - bo[k])]) : INT_MAX;
      }
#pragma unroll
      for (int k = 0; k < kFlatU; k++) {
        const int tr = t0 + k * 32;  // step of lane 0 in this round
        const int q =
            w[k] <= vmax ? find_in_out<MODE>(w[k], Ls, Hs, S, sh, a.adjp + bv, dv) : -1;
        const unsigned hm = __ballot_sync(TR_FULL, q >= 0);
        if (hm == 0) continue;
        const int prior = __shfl_sync(TR_FULL, mycnt, own[k]);
        const int64_t tbase = __shfl_sync(TR_FULL, rb, own[k]);
        const int eo = __shfl_sync(TR_FULL, e, own[k]);
        if (q >= 0) {
          // lanes of this round that walk the same edge: steps [bo, bo + so)
          const int lo = max(bo[k] - tr, 0);
          const unsigned below = hm & lt & ~((1u << lo) - 1u);
          const int64_t euw = (int64_t)eo + 1 + (tr + lane - bo[k]);
          count_hit<MODE>(a, Cs, bv, q, euw, tbase + prior + __popc(below));
        }
        // owners add this round's hits of their own walk
        if (sl > 0) {
          const int lo = P - sl - tr, hi = P - 1 - tr;
          if (hi >= 0 && lo <= 31) {
            const int l0 = max(lo, 0), l1 = min(hi, 31);
            const unsigned seg = (l1 == 31 ? 0xFFFFFFFFu : ((1u << (l1 + 1)) - 1u)) &
                                 ~((1u << l0) - 1u);
            mycnt += __popc(hm & seg);
          }
        }
      }
    }
    if (valid && shrt) {
      if (a.tb) a.cuv[e] = mycnt;
      if (mycnt) atomicAdd(&a.supA[e], mycnt);
    }

    // long walks: the whole warp on one edge, stopping past max out(v)
    unsigned lm = __ballot_sync(TR_FULL, valid && !shrt);
    while (lm) {
      const int o = __ffs(lm) - 1;
      lm &= lm - 1;
      const int eo = __shfl_sync(TR_FULL, e, o);
      const int olen = __shfl_sync(TR_FULL, len, o);
      const int64_t tbase = __shfl_sync(TR_FULL, rb, o);
      const int64_t start = (int64_t)eo + 1;
      int cnt = 0;  // triangles of edge eo so far (warp-uniform)
      for (int t0 = 0; t0 < olen; t0 += 128) {
        int w[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int t = t0 + k * 32 + lane;
          w[k] = t < olen ? __ldg(&a.adjp[start + t]) : INT_MAX;
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const int q =
              w[k] <= vmax ? find_in_out<MODE>(w[k], Ls, Hs, S, sh, a.adjp + bv, dv) : -1;
          const unsigned hm = __ballot_sync(TR_FULL, q >= 0);
          if (q >= 0)
            count_hit<MODE>(a, Cs, bv, q, start + t0 + k * 32 + lane,
                              tbase + cnt + __popc(hm & lt));
          cnt += __popc(hm);
        }
        // out(u) is sorted: past max out(v) nothing can match
        if (__shfl_sync(TR_FULL, w[3], 31) > vmax) break;
      }
      if (lane == 0) {
        if (a.tb) a.cuv[eo] = cnt;
        if (cnt) atomicAdd(&a.supA[eo], cnt);
      }
    }
  }
}

// Warps take equal-cost ranges of inedge round-robin; within a range, each
// head's group is one segment with out(v) staged once.
__global__ void __launch_bounds__(kBlock, 3) k_support_v(SupVArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  unsigned char *base = smem_raw + (size_t)warp * kHeadSmem;
  int32_t *Cs = (int32_t *)base;
  int32_t *Ls = Cs + kHeadCap;
  unsigned short *Hs = (unsigned short *)(Ls + kHeadCap);
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = gw; r < a.P; r += nw) {
    const int64_t ia = __ldg(&a.rb[r]), ib = __ldg(&a.rb[r + 1]);
    int64_t i = ia;
    while (i < ib) {
      const int v = __ldg(&a.ihead[i]);
      const int64_t vbeg = __ldg(&a.inoff[v]), vend = __ldg(&a.inoff[v + 1]);
      const int64_t iend = min(ib, vend);
      const int64_t bv = __ldg(&a.offp[v]);
      const int dv = (int)(__ldg(&a.offp[v + 1]) - bv);
      const int64_t i0 = i;
      i = iend;
      if (dv == 0) continue;  // no w above v: no triangle has v in the middle
      const bool whole = i0 == vbeg && iend == vend;
      if (dv < a.stage_min) {
        // a few entries: search the (L1-cached) global list; staging costs
        // more than the probes of so short a head save
        head_walk<kSearch>(a, i0, iend, bv, dv, __ldg(&a.adjp[bv + dv - 1]), nullptr, nullptr,
                           nullptr, 0, 0);
      } else if (dv <= a.stage_max) {
        int lg = 32 - __clz(max(8 * dv - 1, 63));  // ceil(log2(8 dv)), at least 6
        lg = min(lg, 11);
        const int S = 1 << lg, sh = 32 - lg;
        for (int q = lane; q < dv; q += 32) {
          Ls[q] = __ldg(&a.adjp[bv + q]);
          Cs[q] = 0;
        }
        for (int t = lane; t < S / 2; t += 32) ((uint32_t *)Hs)[t] = 0u;
        __syncwarp();
        for (int q = lane; q < dv; q += 32) {
          unsigned sl = hslot(Ls[q], sh);
          while (atomicCAS(&Hs[sl], (unsigned short)0, (unsigned short)(q + 1)) != 0)
            sl = (sl + 1) & (unsigned)(S - 1);
        }
        __syncwarp();
        head_walk<kStaged>(a, i0, iend, bv, dv, Ls[dv - 1], Ls, Cs, Hs, S, sh);
        __syncwarp();
        for (int q = lane; q < dv; q += 32) {
          if (whole) a.supB[bv + q] = Cs[q];
          else if (Cs[q] != 0) atomicAdd(&a.supB[bv + q], Cs[q]);
        }
        __syncwarp();
      } else if (dv <= a.hash_max) {
        // the warp's whole buffer as a table of 2^lg >= 2 dv position slots
        unsigned short *H2 = (unsigned short *)base;
        int lg = 32 - __clz(2 * dv - 1);
        lg = min(lg, 31 - __clz(kHashOnlyCap * 2));
        const int S = 1 << lg, sh = 32 - lg;
        for (int t = lane; t < S / 2; t += 32) ((uint32_t *)H2)[t] = 0u;
        __syncwarp();
        for (int q = lane; q < dv; q += 32) {
          unsigned sl = hslot(__ldg(&a.adjp[bv + q]), sh);
          while (atomicCAS(&H2[sl], (unsigned short)0, (unsigned short)(q + 1)) != 0)
            sl = (sl + 1) & (unsigned)(S - 1);
        }
        __syncwarp();
        head_walk<kHashOnly>(a, i0, iend, bv, dv, __ldg(&a.adjp[bv + dv - 1]), nullptr,
                             nullptr, H2, S, sh);
        __syncwarp();
      } else {
        head_walk<kSearch>(a, i0, iend, bv, dv, __ldg(&a.adjp[bv + dv - 1]), nullptr, nullptr,
                           nullptr, 0, 0);
      }
    }
  }
}

// Edges grouped by head: counts, then a fill with one cursor per head.
__global__ void k_head_count(int64_t m, const int32_t *adjp, unsigned long long *cnt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[adjp[e]], 1ull);
}

__global__ void k_seq(int64_t m, int32_t *x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    x[e] = (int32_t)e;
}

// Head-centric walk cost of inedge[i] = (u, v): |out(u) after v| plus the
// fixed per-edge cost; and, per edge id, the most triangles it can close as
// e_uv, min(|out(v)|, |out(u) after v|) (its record region).
__global__ void k_walk_cost_v(int64_t m, const int64_t *offp, const int32_t *adjp,
                              const int32_t *esrc, const int32_t *inedge, int64_t *cost,
                              int64_t *bound, int edge_cost) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= m;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i == m) {
      cost[m] = 0;
      bound[m] = 0;
      continue;
    }
    const int e = inedge[i];
    const int64_t after = offp[esrc[e] + 1] - (int64_t)e - 1;
    cost[i] = after + edge_cost;
    const int v = adjp[i];
    const int64_t dv = offp[v + 1] - offp[v];
    const int u = esrc[i];
    const int64_t after_i = offp[u + 1] - i - 1;
    bound[i] = min(dv, after_i);
  }
}

// The list walk: warps take equal-cost ranges of oriented edges round-robin.
// list(e)'s first supA[e] entries come from the walk of e's tail (cursors in
// shared memory when one warp walks all of the tail's out-list, else the
// global cursors curA), the rest from the global cursors curB.
__global__ void __launch_bounds__(kBlock, 4) k_list_walk(ListArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = lane_id();
  unsigned char *base = smem_raw + (size_t)warp * kListSmem;
  // layout: cursors (8-byte aligned first), then L, then the out(v) chunk
  unsigned long long *Cs = (unsigned long long *)base;
  int32_t *Ls = (int32_t *)(base + (size_t)kListCap * 8);
  int32_t *Abuf = Ls + kListCap;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = gw; r < a.P; r += nw) {
    const int64_t ea = __ldg(&a.rb[r]), eb = __ldg(&a.rb[r + 1]);
    int64_t e = ea;
    while (e < eb) {
      const int u = __ldg(&a.esrc[e]);
      const int64_t bu = __ldg(&a.offp[u]);
      const int d = (int)(__ldg(&a.offp[u + 1]) - bu);
      const int i0 = (int)(e - bu);
      const int iend = (int)(min(eb, bu + d) - bu);
      e = bu + iend;
      const int i1 = min(iend, d - 1);  // the last out-neighbour closes no triangle here
      if (i0 >= i1) continue;
      const bool whole = i0 == 0 && iend >= d - 1;  // this warp walks all of out(u)
      if (d <= a.stage_max) {
        for (int q = lane; q < d; q += 32) {
          Ls[q] = __ldg(&a.adjp[bu + q]);
          Cs[q] = (unsigned long long)__ldg(&a.curA[bu + q]);
        }
        __syncwarp();
        OutList<true> ol{Ls, d};
        walk<true>(a, bu, ol, whole ? Cs : a.curA + bu, i0, i1, Abuf);
      } else {
        OutList<false> ol{a.adjp + bu, d};
        walk<false>(a, bu, ol, a.curA + bu, i0, i1, Abuf);
      }
      __syncwarp();
    }
  }
}

// Walk cost of each oriented edge: |out(v)| for (u, v) unless v is the last
// entry of out(u), plus `edge_cost` for every edge; and the most triangles
// (u, v, w) it can close, min(|out(v)|, entries of out(u) after v).  The
// fixed part stands for what a warp pays per edge whatever the lists: the
// offsets it loads and, for owners with a single out-edge (the long run of
// degree-1 vertices at the bottom of the degree order), the step to the
// next owner.  Without it that run is free and falls into one range, which
// one warp then steps through owner by owner.
__global__ void k_walk_cost(int64_t m, const int64_t *offp, const int32_t *adjp,
                            const int32_t *esrc, int64_t *cost, int64_t *bound, int edge_cost) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = 0, b = 0;
    if (e < m) {
      const int u = esrc[e];
      const int64_t end = offp[u + 1];
      c = edge_cost;
      if (e != end - 1) {
        const int v = adjp[e];
        const int64_t a = offp[v + 1] - offp[v];
        b = min(a, end - 1 - e);
        c += a;
      }
    }
    cost[e] = c;
    bound[e] = b;
  }
}

// Dense triangle lists from the records, in two passes.  The first cuv[x]
// entries of edge x's list are the triangles x closes as the walked edge, in
// record order: its records themselves, which stay where the walk wrote
// them, unless the full lists are asked for (then they are copied to
// pairs[toff[x] ..)).  The rest are handed out from x's cursor cur[x] (set
// to the first slot after the own part).
//
// Pass 1 (k_lists_owner) writes, for each record (e_uw, e_vw) of walked edge
// e_uv, e_uw's entry (e_uv, e_vw) (and, for the full lists, e_uv's own
// entry).  e_uw lies in out(u), so every cursor pass 1 touches for the
// records of u's out-edges is one of u's out-edges.  Pass 2 (k_lists_head)
// writes e_vw's entry (e_uv, e_uw); e_vw lies in out(v), so the records of
// v's in-edges touch only cursors of v's out-edges.  Each pass therefore
// splits the vertices (owners u, heads v) into ranges of about equal record
// counts, and one block takes a whole range: the cursors of the range's
// out-edges (at most a few thousand, since in degree order an out-degree d
// needs d neighbours of degree >= d) are counted in shared memory, with no
// global atomic, and each range's list writes land in the range's own
// stretch of `pairs`, which L2 merges into whole sectors.  A range with more
// out-edges than the shared counters hold (a vertex of huge out-degree)
// falls back to global atomics on its cursors.  Pass 1 adds its counts to
// the cursors at the end of each range, so pass 2 continues after them.
//
// Within a range the warps claim chunks of consecutive edges (pass 1) or
// in-edges (pass 2) from a shared counter, and walk a chunk's records 4 per
// lane per step, so that 4 record loads are in flight per lane before any
// store needs them.  A chunk holds up to 32 edges, fewer in a range whose
// edges carry many records (about 256 records per chunk), so that a range
// of a few heavy edges still keeps every warp of the block busy.
constexpr int kListU = 4;
constexpr int kLBlock = 512;
constexpr int kLCap = 16384;       // shared cursor counters per range (64 KB)
constexpr int kLEdgeCost = 4;      // range cost per edge (next to its records)
constexpr int64_t kLRangeCost = (int64_t)kLCap * kLEdgeCost / 2;

struct ListPass {
  int64_t m, n;
  const int64_t *offp;
  const int64_t *tbpre;
  const int2 *tb;
  const int32_t *cuv;
  const int64_t *toff;        // pass 1, whole lists: own slots; null with own parts in place
  unsigned long long *cur;    // per edge: next free slot of its rest part
  const int32_t *inedge;      // pass 2: edges grouped by head
  const int64_t *inoff;
  const int64_t *vb;          // range r = vertices [vb[r], vb[r+1])
  const int64_t *pre;         // exclusive prefix of (records + kLEdgeCost) over the walk order
  int64_t nranges;
  unsigned long long *next;   // range counter
  int2 *pairs;
  uint32_t *tids;
  int64_t entries;
  int *err;
};

__device__ __forceinline__ void pairs_store(const ListPass &a, int64_t x, int2 v, uint32_t tid) {
  a.pairs[x] = v;
  if (a.tids) a.tids[x] = tid;
}

// One range of a pass; HEAD = pass 2.  Every thread of the block calls it.
template <bool HEAD>
__device__ __forceinline__ void list_range(const ListPass &a, int64_t v0, int64_t v1,
                                           int *s_ctr, int *s_next) {
  const int lane = lane_id();
  const int64_t e0 = a.offp[v0], e1 = a.offp[v1], ne = e1 - e0;
  const bool local = ne <= kLCap;
  if (local)
    for (int64_t i = threadIdx.x; i < ne; i += blockDim.x) s_ctr[i] = 0;
  if (threadIdx.x == 0) *s_next = 0;
  __syncthreads();
  // pass 1 walks the edges [e0, e1); pass 2 the in-edges of the heads
  const int64_t w0 = HEAD ? a.inoff[v0] : e0, w1 = HEAD ? a.inoff[v1] : e1;
  const int64_t recs = a.pre[w1] - a.pre[w0] - kLEdgeCost * (w1 - w0);
  const int64_t cw = (256 * (w1 - w0)) / (recs > 0 ? recs : 1);
  const int chunk = cw < 1 ? 1 : cw > 32 ? 32 : (int)cw;
  for (;;) {
    int ci = 0;
    if (lane == 0) ci = atomicAdd(s_next, 1);
    ci = __shfl_sync(TR_FULL, ci, 0);
    const int64_t base = w0 + (int64_t)ci * chunk;
    if (base >= w1) break;
    const int64_t i = base + lane;
    const bool in = lane < chunk && i < w1;
    const int e = in ? (HEAD ? __ldg(&a.inedge[i]) : (int)i) : 0;
    const int c = in ? __ldg(&a.cuv[e]) : 0;
    const int64_t r0 = in ? __ldg(&a.tbpre[e]) : 0;
    const int64_t l0 = (!HEAD && in && a.toff) ? __ldg(&a.toff[e]) : 0;
    const int P = warp_incl_scan(c);
    const int total = __shfl_sync(TR_FULL, P, 31);
    for (int t0 = 0; t0 < total; t0 += 32 * kListU) {
      int2 rec[kListU];
      int64_t x1[kListU], x2[kListU];
      int eo[kListU];
      uint32_t ri[kListU];  // record index = triangle id
#pragma unroll
      for (int k = 0; k < kListU; k++) {
        const int t = t0 + k * 32 + lane;
        const int o = warp_owner(P, t < total ? t : total - 1);
        const int64_t orr = __shfl_sync(TR_FULL, r0, o);
        const int64_t ol = __shfl_sync(TR_FULL, l0, o);
        const int oP = __shfl_sync(TR_FULL, P, o), oc = __shfl_sync(TR_FULL, c, o);
        eo[k] = __shfl_sync(TR_FULL, e, o);
        const int j = t - (oP - oc);
        x1[k] = ol + j;
        ri[k] = (uint32_t)(orr + j);
        rec[k] = t < total ? __ldg(&a.tb[orr + j]) : make_int2(-1, -1);  // (e_uw, e_vw)
      }
#pragma unroll
      for (int k = 0; k < kListU; k++) {
        const int f = HEAD ? rec[k].y : rec[k].x;  // the edge whose cursor hands out the slot
        x2[k] = 0;
        if (f < 0) continue;
        const int64_t fi = (int64_t)f - e0;
        if (fi < 0 || fi >= ne) {
          atomicExch(a.err, TRUSS_ECHECK);  // a record outside its range: skip it
          rec[k] = make_int2(-1, -1);
          continue;
        }
        x2[k] = local ? (int64_t)a.cur[f] + atomicAdd(&s_ctr[fi], 1)
                      : (int64_t)atomicAdd(&a.cur[f], 1ull);
      }
#pragma unroll
      for (int k = 0; k < kListU; k++) {
        if (rec[k].x < 0) continue;
        const bool own = !HEAD && a.toff;
        if ((!own || x1[k] < a.entries) && x2[k] < a.entries) {
          if (own) pairs_store(a, x1[k], rec[k], ri[k]);
          pairs_store(a, x2[k], HEAD ? make_int2(eo[k], rec[k].x) : make_int2(eo[k], rec[k].y),
                      ri[k]);
        } else {
          atomicExch(a.err, TRUSS_ECHECK);
        }
      }
    }
  }
  __syncthreads();
  // pass 1: later passes continue after this range's slots
  if (!HEAD && local)
    for (int64_t i = threadIdx.x; i < ne; i += blockDim.x) a.cur[e0 + i] += (unsigned)s_ctr[i];
}

template <bool HEAD>
__global__ void __launch_bounds__(kLBlock, 2) k_lists_pass(ListPass a) {
  extern __shared__ int s_ctr[];
  __shared__ long long s_r;
  __shared__ int s_next;
  for (;;) {
    if (threadIdx.x == 0) s_r = (long long)atomicAdd(a.next, 1ull);
    __syncthreads();
    const int64_t r = s_r;
    if (r >= a.nranges) return;
    const int64_t v0 = a.vb[r], v1 = a.vb[r + 1];
    if (v0 < v1) list_range<HEAD>(a, v0, v1, s_ctr, &s_next);  // ends with a block barrier
    else __syncthreads();
  }
}

// Range costs of the two passes: pass 1 per edge e (grouped by owner),
// cuv[e] + kLEdgeCost; pass 2 per in-edge position i, cuv[inedge[i]] +
// kLEdgeCost (and kLEdgeCost per out-edge of each head, added below).
__global__ void k_list_costs(int64_t m, const int32_t *cuv, const int32_t *inedge, int64_t *c1,
                             int64_t *c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= m;
       i += (int64_t)gridDim.x * blockDim.x) {
    c1[i] = i < m ? (int64_t)cuv[i] + kLEdgeCost : 0;
    c2[i] = i < m ? (int64_t)cuv[inedge[i]] + kLEdgeCost : 0;
  }
}

// vb[r] = first vertex v with cost(v) >= r * kLRangeCost, for r < nr, and
// vb[nr] = n; cost(v) = pre[idx[v]] (+ kLEdgeCost * offp[v] for pass 2).
__global__ void k_list_ranges(int64_t n, int64_t nr, const int64_t *pre, const int64_t *idx,
                              const int64_t *offp, bool head, int64_t *vb) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= nr;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (r == nr) {
      vb[r] = n;
      continue;
    }
    const int64_t x = r * kLRangeCost;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      const int64_t c = pre[idx[mid]] + (head ? kLEdgeCost * offp[mid] : 0);
      if (c < x) lo = mid + 1; else hi = mid;
    }
    vb[r] = lo;
  }
}

// Cursors for the list passes: the first slot after each edge's own part
// (base = toff and skip = cuv for the full lists, base = the rest offsets
// and skip = null with the own parts in place).
__global__ void k_cursors_rec(int64_t m, const int64_t *base, const int32_t *skip,
                              unsigned long long *cur) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    cur[e] = (unsigned long long)(base[e] + (skip ? skip[e] : 0));
}

// Length of each edge's rest part, sup - cuv (and 0 at e = m, so that the
// exclusive sum ends with the total).
__global__ void k_rest_len(int64_t m, const int32_t *sup, const int32_t *cuv, int64_t *len) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= m;
       e += (int64_t)gridDim.x * blockDim.x)
    len[e] = e < m ? (int64_t)(sup[e] - cuv[e]) : 0;
}

__global__ void k_sum(int64_t m, const int32_t *supA, const int32_t *supB, int32_t *sup,
                      int64_t *sup64) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= m;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < m) {
      int32_t s = supA[e] + supB[e];
      sup[e] = s;
      sup64[e] = s;
    } else {
      sup64[e] = 0;
    }
  }
}

// List cursors: e's owner part starts at toff[e], its other part at
// toff[e] + supA[e].
__global__ void k_cursors(int64_t m, const int64_t *toff, const int32_t *supA,
                          unsigned long long *curA, unsigned long long *curB) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    curA[e] = (unsigned long long)toff[e];
    curB[e] = (unsigned long long)(toff[e] + supA[e]);
  }
}

// rb[r] = first position whose walk-cost prefix reaches r W / P, for
// r = 0 .. P: one search per range here instead of two dependent chains of
// ~log2(m) loads at the start of every range in a walk.
__global__ void k_range_bounds(int64_t m, int64_t P, int64_t W, const int64_t *wpre,
                               int64_t *rb) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= P;
       r += (int64_t)gridDim.x * blockDim.x)
    rb[r] = lower_bound64(wpre, m, range_point(W, P, r));
}

// The owner-centric list walk, used when the triangle records do not fit.
int launch_list_walk(Arena &A, ListArgs a, const SupportCfg &cfg, cudaStream_t s) {
  int dev = 0, sms = cfg.sms;
  TR_CUDA(cudaGetDevice(&dev));
  if (sms <= 0) TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t smem = (size_t)(kBlock / 32) * kListSmem;
  // the per-warp buffers exceed the default 48 KB window: opt in to the
  // larger per-block limit
  TR_CUDA(cudaFuncSetAttribute(k_list_walk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  int occ = 0;
  TR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_list_walk, kBlock, smem));
  if (occ < 1) occ = 1;
  const int grid = sms * occ;
  const int64_t warps = (int64_t)grid * (kBlock / 32);
  int64_t P = a.W / (cfg.range_work > 0 ? cfg.range_work : kRangeWork);
  if (P < warps) P = warps;
  if (P > a.m) P = a.m > 0 ? a.m : 1;
  a.P = P;
  int64_t *rb = A.get<int64_t>(P + 1);
  if (!rb) return TRUSS_ENOMEM;
  k_range_bounds<<<grid_for(P + 1, 256, 152 * 8), 256, 0, s>>>(a.m, P, a.W, a.wpre, rb);
  TR_LAUNCHED();
  a.rb = rb;
  a.stage_max = cfg.stage_max > 0 && cfg.stage_max < kListCap ? cfg.stage_max : kListCap;
  k_list_walk<<<grid, kBlock, smem, s>>>(a);
  TR_LAUNCHED();
  return TRUSS_OK;
}

int launch_walk_v(Arena &A, SupVArgs a, const SupportCfg &cfg, cudaStream_t s) {
  int dev = 0, sms = cfg.sms;
  TR_CUDA(cudaGetDevice(&dev));
  if (sms <= 0) TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t smem = (size_t)(kBlock / 32) * kHeadSmem;
  TR_CUDA(cudaFuncSetAttribute(k_support_v, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  int occ = 0;
  TR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_support_v, kBlock, smem));
  if (occ < 1) occ = 1;
  const int grid = sms * occ;
  const int64_t warps = (int64_t)grid * (kBlock / 32);
  int64_t P = a.W / (cfg.range_work > 0 ? cfg.range_work : kRangeWork);
  if (P < warps) P = warps;
  if (P > a.m) P = a.m > 0 ? a.m : 1;
  a.P = P;
  int64_t *rb = A.get<int64_t>(P + 1);
  if (!rb) return TRUSS_ENOMEM;
  k_range_bounds<<<grid_for(P + 1, 256, 152 * 8), 256, 0, s>>>(a.m, P, a.W, a.wpre, rb);
  TR_LAUNCHED();
  a.rb = rb;
  a.stage_max = cfg.stage_max > 0 && cfg.stage_max < kHeadCap ? cfg.stage_max : kHeadCap;
  a.hash_max = kHashOnlyCap;
  a.stage_min = kStageMin;
  k_support_v<<<grid, kBlock, smem, s>>>(a);
  TR_LAUNCHED();
  return TRUSS_OK;
}

}  // namespace

int run_support(Arena &A, const Csr &g, const SupportCfg &cfg, SupportOut *out, cudaStream_t s) {
  const int64_t m = g.m, n = g.n;
  int32_t *supA = A.get<int32_t>(m), *supB = A.get<int32_t>(m), *sup = A.get<int32_t>(m);
  int64_t *sup64 = A.get<int64_t>(m + 1), *toff = A.get<int64_t>(m + 1);
  int64_t *wcost = A.get<int64_t>(m + 1), *wpre = A.get<int64_t>(m + 1);
  int64_t *wbound = A.get<int64_t>(m + 1), *tbpre = A.get<int64_t>(m + 1);
  unsigned long long *hcnt = A.get<unsigned long long>(n + 1);
  int64_t *inoff = A.get<int64_t>(n + 1);
  int32_t *inedge = A.get<int32_t>(m), *ihead = A.get<int32_t>(m);
  if (!supA || !supB || !sup || !sup64 || !toff || !wcost || !wpre || !wbound || !tbpre ||
      !hcnt || !inoff || !inedge || !ihead)
    return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(supA, 0, sizeof(int32_t) * m, s));
  TR_CUDA(cudaMemsetAsync(supB, 0, sizeof(int32_t) * m, s));
  int64_t W = 0, R = 0;
  if (m > 0) {
    // edges grouped by head: counts and their prefix give each head's
    // group; a stable radix sort of (head, edge id) fills the groups in
    // edge order (the edge ids sit in wcost's memory until the sort)
    TR_CUDA(cudaMemsetAsync(hcnt, 0, sizeof(unsigned long long) * (n + 1), s));
    k_head_count<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, g.adjp, hcnt);
    TR_LAUNCHED();
    int32_t *ids = (int32_t *)wcost;
    k_seq<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, ids);
    TR_LAUNCHED();
    const int hbits = bits_for((uint64_t)(n > 1 ? n - 1 : 1));
    size_t tb = 0, tb2 = 0, tb3 = 0;
    TR_TRY(exclusive_sum_i64(nullptr, &tb, (const int64_t *)hcnt, inoff, n + 1, s));
    TR_TRY(exclusive_sum_i64(nullptr, &tb2, wcost, wpre, m + 1, s));
    TR_TRY(sort_pairs_u32(nullptr, &tb3, (const uint32_t *)g.adjp, (uint32_t *)ihead, ids, inedge,
                          m, 0, hbits, s));
    tb2 = tb2 > tb ? tb2 : tb;
    tb2 = tb2 > tb3 ? tb2 : tb3;
    void *tmp = A.alloc(tb2);
    if (!tmp) return TRUSS_ENOMEM;
    TR_TRY(exclusive_sum_i64(tmp, &tb, (const int64_t *)hcnt, inoff, n + 1, s));
    TR_TRY(sort_pairs_u32(tmp, &tb3, (const uint32_t *)g.adjp, (uint32_t *)ihead, ids, inedge, m,
                          0, hbits, s));
    const int ec = cfg.pair_cost > 0 ? cfg.pair_cost : cfg.pair_cost < 0 ? 0 : kEdgeCost;
    k_walk_cost_v<<<grid_for(m + 1, 256, 152 * 16), 256, 0, s>>>(m, g.offp, g.adjp, g.esrc,
                                                                  inedge, wcost, wbound, ec);
    TR_LAUNCHED();
    TR_TRY(exclusive_sum_i64(tmp, &tb2, wcost, wpre, m + 1, s));
    if (cfg.records) TR_TRY(exclusive_sum_i64(tmp, &tb2, wbound, tbpre, m + 1, s));
    TR_CUDA(cudaMemcpyAsync(&W, wpre + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (cfg.records)
      TR_CUDA(cudaMemcpyAsync(&R, tbpre + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TR_CUDA(cudaStreamSynchronize(s));
  }
  // Records need 8 R bytes now, and the lists later 24 bytes per triangle
  // when they are whole, 16 with the own parts left in the records, plus a
  // few words per edge for the list passes and the peel.  The walk records
  // only if the lists fit at their bound (a triangle per record slot, T <=
  // R); otherwise the list pass walks the graph a second time.  Whole lists
  // or own parts in place is decided after the walk, from the exact
  // triangle count (the bound can be twice the count or more).
  int2 *recs = nullptr;
  int32_t *cuv = nullptr;
  bool in_place = false;
  if (cfg.records && R > 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      fr = 0;
    }
    const double avail = (double)A.headroom(fr);
    const double need_whole = 1.05 * (32.0 * (double)R + 20.0 * (double)m);
    const double need_in_place = 1.05 * (24.0 * (double)R + 36.0 * (double)m);
    const bool use = cfg.full_lists ? need_whole < avail : need_in_place < avail;
    if (use) {
      recs = A.get<int2>(R);
      cuv = A.get<int32_t>(m);
      if (!recs || !cuv) {
        recs = nullptr;
        cuv = nullptr;
      } else {
        TR_CUDA(cudaMemsetAsync(cuv, 0, sizeof(int32_t) * m, s));
      }
    }
  }
  if (W > 0) {
    SupVArgs a{};
    a.n = n;
    a.m = m;
    a.offp = g.offp;
    a.adjp = g.adjp;
    a.esrc = g.esrc;
    a.inedge = inedge;
    a.ihead = ihead;
    a.inoff = inoff;
    a.wcost = wcost;
    a.wpre = wpre;
    a.W = W;
    a.ecost = cfg.pair_cost > 0 ? cfg.pair_cost : cfg.pair_cost < 0 ? 0 : kEdgeCost;
    a.supA = supA;
    a.supB = supB;
    a.tbpre = tbpre;
    a.tb = recs;
    a.cuv = cuv;
    TR_TRY(launch_walk_v(A, a, cfg, s));
  }
  k_sum<<<grid_for(m + 1, 256, 152 * 16), 256, 0, s>>>(m, supA, supB, sup, sup64);
  TR_LAUNCHED();
  size_t tb = 0;
  TR_TRY(exclusive_sum_i64(nullptr, &tb, sup64, toff, m + 1, s));
  void *tmp = A.alloc(tb);
  if (!tmp) return TRUSS_ENOMEM;
  TR_TRY(exclusive_sum_i64(tmp, &tb, sup64, toff, m + 1, s));
  int64_t total = 0;
  TR_CUDA(cudaMemcpyAsync(&total, toff + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  out->sup = sup;
  out->supA = supA;
  out->toff = toff;
  out->walk = W;
  out->entries = total;
  out->inedge = inedge;
  out->inoff = inoff;
  if (recs && !cfg.full_lists) {
    if (cfg.in_place) {
      in_place = true;
    } else {
      // whole lists: 3T entries, the peel's work items (up to 3T/16 + m, two
      // queues) and about 100 B per edge for the list passes and the peel
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        fr = 0;
      }
      const double tri = (double)(total / 3);
      in_place = !(1.05 * (30.0 * tri + 100.0 * (double)m) < (double)A.headroom(fr));
    }
  }
  out->tbpre = recs ? tbpre : nullptr;
  out->records = recs ? R : 0;
  out->tb = recs;
  out->cuv = recs ? cuv : nullptr;
  out->in_place = recs && in_place;
  return TRUSS_OK;
}

int run_lists(Arena &A, const Csr &g, const SupportCfg &cfg, const SupportOut &so, int2 *pairs,
              uint32_t *tids, TriLists *out, cudaStream_t s) {
  const int64_t m = g.m;
  *out = TriLists{};
  out->rest = pairs;
  out->off = so.toff;
  if (m == 0 || so.entries == 0) return TRUSS_OK;
  if (so.tb) {
    const bool in_place = so.in_place;
    if (tids && in_place) return TRUSS_EINVAL;  // triangle ids come with whole lists
    unsigned long long *cur = A.get<unsigned long long>(m);
    int *err = A.get<int>(1);
    if (!cur || !err) return TRUSS_ENOMEM;
    TR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    const int64_t rest = list_rest_entries(so);
    if (in_place) {
      int64_t *len = A.get<int64_t>(m + 1), *roff = A.get<int64_t>(m + 1);
      if (!len || !roff) return TRUSS_ENOMEM;
      k_rest_len<<<grid_for(m + 1, 256, 152 * 16), 256, 0, s>>>(m, so.sup, so.cuv, len);
      TR_LAUNCHED();
      size_t tb = 0;
      TR_TRY(exclusive_sum_i64(nullptr, &tb, len, roff, m + 1, s));
      void *tmp = A.alloc(tb);
      if (!tmp) return TRUSS_ENOMEM;
      TR_TRY(exclusive_sum_i64(tmp, &tb, len, roff, m + 1, s));
      k_cursors_rec<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, roff, nullptr, cur);
      TR_LAUNCHED();
      out->own = so.tb;
      out->own_off = so.tbpre;
      out->own_cnt = so.cuv;
      out->off = roff;
    } else {
      k_cursors_rec<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, so.toff, so.cuv, cur);
      TR_LAUNCHED();
    }
    // vertex ranges of about kLRangeCost: pass 1 over owners (edge order),
    // pass 2 over heads (the support walk's in-edge index)
    const int64_t n = g.n, tri = so.entries / 3;
    int64_t *c1 = A.get<int64_t>(m + 1), *c2 = A.get<int64_t>(m + 1);
    int64_t *p1 = A.get<int64_t>(m + 1), *p2 = A.get<int64_t>(m + 1);
    const int64_t nr1 = (tri + kLEdgeCost * m) / kLRangeCost + 1;
    const int64_t nr2 = (tri + 2 * kLEdgeCost * m) / kLRangeCost + 1;
    int64_t *vb1 = A.get<int64_t>(nr1 + 1), *vb2 = A.get<int64_t>(nr2 + 1);
    unsigned long long *next = A.get<unsigned long long>(2);
    if (!c1 || !c2 || !p1 || !p2 || !vb1 || !vb2 || !next) return TRUSS_ENOMEM;
    k_list_costs<<<grid_for(m + 1, 256, 152 * 16), 256, 0, s>>>(m, so.cuv, so.inedge, c1, c2);
    TR_LAUNCHED();
    size_t tb = 0;
    TR_TRY(exclusive_sum_i64(nullptr, &tb, c1, p1, m + 1, s));
    void *tmp = A.alloc(tb);
    if (!tmp) return TRUSS_ENOMEM;
    TR_TRY(exclusive_sum_i64(tmp, &tb, c1, p1, m + 1, s));
    TR_TRY(exclusive_sum_i64(tmp, &tb, c2, p2, m + 1, s));
    k_list_ranges<<<grid_for(nr1 + 1, 256, 152 * 8), 256, 0, s>>>(n, nr1, p1, g.offp, g.offp,
                                                                    false, vb1);
    TR_LAUNCHED();
    k_list_ranges<<<grid_for(nr2 + 1, 256, 152 * 8), 256, 0, s>>>(n, nr2, p2, so.inoff, g.offp,
                                                                    true, vb2);
    TR_LAUNCHED();
    TR_CUDA(cudaMemsetAsync(next, 0, 2 * sizeof(unsigned long long), s));
    int dev = 0, sms = cfg.sms;
    TR_CUDA(cudaGetDevice(&dev));
    if (sms <= 0) TR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = sizeof(int) * kLCap;
    TR_CUDA(cudaFuncSetAttribute(k_lists_pass<false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TR_CUDA(cudaFuncSetAttribute(k_lists_pass<true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    TR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lists_pass<false>, kLBlock,
                                                          smem));
    if (occ < 1) occ = 1;
    ListPass lp{};
    lp.m = m;
    lp.n = n;
    lp.offp = g.offp;
    lp.tbpre = so.tbpre;
    lp.tb = so.tb;
    lp.cuv = so.cuv;
    lp.toff = in_place ? nullptr : so.toff;
    lp.cur = cur;
    lp.inedge = so.inedge;
    lp.inoff = so.inoff;
    lp.pairs = pairs;
    lp.tids = tids;
    lp.entries = rest;
    lp.err = err;
    lp.vb = vb1;
    lp.pre = p1;
    lp.nranges = nr1;
    lp.next = next;
    k_lists_pass<false><<<sms * occ, kLBlock, smem, s>>>(lp);
    TR_LAUNCHED();
    lp.vb = vb2;
    lp.pre = p2;
    lp.nranges = nr2;
    lp.next = next + 1;
    k_lists_pass<true><<<sms * occ, kLBlock, smem, s>>>(lp);
    TR_LAUNCHED();
    int h_err = 0;
    TR_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TR_CUDA(cudaStreamSynchronize(s));
    return h_err != 0 ? TRUSS_ECHECK : TRUSS_OK;
  }
  // No records (short of memory): walk the graph again, owner by owner, and
  // write the lists directly.  Its ranges need the owner-centric walk cost.
  unsigned long long *curA = A.get<unsigned long long>(m), *curB = A.get<unsigned long long>(m);
  int64_t *wcost = A.get<int64_t>(m + 1), *wpre = A.get<int64_t>(m + 1);
  int64_t *wbound = A.get<int64_t>(m + 1);
  int *err = A.get<int>(1);
  if (!curA || !curB || !wcost || !wpre || !wbound || !err) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  const int ec = cfg.pair_cost > 0 ? cfg.pair_cost : cfg.pair_cost < 0 ? 0 : kEdgeCost;
  k_walk_cost<<<grid_for(m + 1, 256, 152 * 16), 256, 0, s>>>(m, g.offp, g.adjp, g.esrc, wcost,
                                                              wbound, ec);
  TR_LAUNCHED();
  size_t tb = 0;
  TR_TRY(exclusive_sum_i64(nullptr, &tb, wcost, wpre, m + 1, s));
  void *tmp = A.alloc(tb);
  if (!tmp) return TRUSS_ENOMEM;
  TR_TRY(exclusive_sum_i64(tmp, &tb, wcost, wpre, m + 1, s));
  int64_t W = 0;
  TR_CUDA(cudaMemcpyAsync(&W, wpre + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  k_cursors<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(m, so.toff, so.supA, curA, curB);
  TR_LAUNCHED();
  ListArgs a{};
  a.n = g.n;
  a.m = m;
  a.offp = g.offp;
  a.adjp = g.adjp;
  a.esrc = g.esrc;
  a.wpre = wpre;
  a.W = W;
  a.curA = curA;
  a.curB = curB;
  a.pairs = pairs;
  a.entries = so.entries;
  a.err = err;
  TR_TRY(launch_list_walk(A, a, cfg, s));
  int h_err = 0;
  TR_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  return h_err != 0 ? TRUSS_ECHECK : TRUSS_OK;
}

}  // namespace tr

namespace tr {

namespace {

// Algorithmic bytes of the head-centric walk, summed over vertices w (the
// out-degree d = |out(w)|): as a head, out(w) is staged and its counts are
// stored (16 + 8d, when d >= 1); as a tail, each out-edge at position i
// costs its index, tail and offsets (24 B) and the read of the d - i - 1
// entries after it (4 B each), 24d + 2d(d-1) in all.
__global__ void k_count_walk(int64_t n, const int64_t *offp, unsigned long long *acc) {
  unsigned long long local = 0;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n;
       w += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long d = (unsigned long long)(offp[w + 1] - offp[w]);
    if (d == 0) continue;
    local += 16ull + 8ull * d + 24ull * d + 2ull * d * (d - 1);
  }
  for (int o = 16; o >= 1; o >>= 1) local += __shfl_down_sync(TR_FULL, local, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, local);
}
// Algorithmic bytes of the owner-centric list walk: per owner u of
// out-degree d >= 2, its offsets, out(u) and its cursors (16 + 8d); per
// walked edge (u, v), v's offsets and out(v) (16 + 4 |out(v)|).
__global__ void k_count_list_walk(int64_t n, const int64_t *offp, const int32_t *adjp,
                                  unsigned long long *acc) {
  unsigned long long local = 0;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t bu = offp[u], d = offp[u + 1] - bu;
    if (d < 2) continue;
    local += 16ull + 8ull * (unsigned long long)d;
    for (int64_t i = 0; i < d - 1; i++) {
      const int v = adjp[bu + i];
      local += 16ull + 4ull * (unsigned long long)(offp[v + 1] - offp[v]);
    }
  }
  for (int o = 16; o >= 1; o >>= 1) local += __shfl_down_sync(TR_FULL, local, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, local);
}
// Sum over the oriented edges (u, v) of d+(u) + d+(v): the out-list entries
// a forward merge of out(u) and out(v) reads for every edge.
__global__ void k_count_merge(int64_t m, const int64_t *offp, const int32_t *esrc,
                              const int32_t *adjp, unsigned long long *acc) {
  unsigned long long local = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int u = esrc[e], v = adjp[e];
    local += (unsigned long long)(offp[u + 1] - offp[u] + offp[v + 1] - offp[v]);
  }
  for (int o = 16; o >= 1; o >>= 1) local += __shfl_down_sync(TR_FULL, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(acc, local);
}
}  // namespace

// Algorithmic bytes of the support pass.  b_sup: 4 B per out-list entry of
// the forward merge of every oriented edge, 32 B of offsets, 8 B of
// endpoints and a 4-B support write per edge, and three 8-B read-modify-
// writes per triangle.  b_sup_design: the walk this library runs (above)
// plus, per triangle, the read-modify-write of e_uw's count (8 B) and, when
// recording, its 8-B record.  Of the list pass: see below.
int count_support_bytes(Arena &A, const Csr &g, int64_t triangles, bool records, bool in_place,
                        double *b_sup, double *b_sup_design, double *b_lists, cudaStream_t s) {
  unsigned long long *acc = A.get<unsigned long long>(2);
  if (!acc) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), s));
  unsigned long long hm = 0;
  if (g.m > 0) {
    k_count_merge<<<grid_for(g.m, 256, 152 * 8), 256, 0, s>>>(g.m, g.offp, g.esrc, g.adjp,
                                                               acc + 1);
    TR_LAUNCHED();
    TR_CUDA(cudaMemcpyAsync(&hm, acc + 1, sizeof(hm), cudaMemcpyDeviceToHost, s));
  }
  if (g.n > 0 && g.m > 0) {
    k_count_walk<<<grid_for(g.n, 256, 152 * 8), 256, 0, s>>>(g.n, g.offp, acc);
    TR_LAUNCHED();
  }
  unsigned long long h = 0, hl = 0;
  TR_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  if (!records && g.n > 0 && g.m > 0) {
    TR_CUDA(cudaMemsetAsync(acc, 0, sizeof(unsigned long long), s));
    k_count_list_walk<<<grid_for(g.n, 256, 152 * 8), 256, 0, s>>>(g.n, g.offp, g.adjp, acc);
    TR_LAUNCHED();
    TR_CUDA(cudaMemcpyAsync(&hl, acc, sizeof(hl), cudaMemcpyDeviceToHost, s));
    TR_CUDA(cudaStreamSynchronize(s));
  }
  // whole lists from records: the record read by both passes, three
  // entries, two cursor RMWs (56 B per triangle), and per edge the cursor
  // set-up and both passes' offset/count reads (56 B; the head-order sort is
  // not counted).  Own parts in place: two entries (48 B per triangle), and
  // per edge the rest lengths and their scan (32 B), the cursor set-up
  // (16 B) and both passes' reads (28 B).  Lists by a second walk: the walk
  // again plus 60 B per triangle.
  *b_sup = 4.0 * (double)hm + 44.0 * (double)g.m + 24.0 * (double)triangles;
  *b_sup_design = (double)h + (records ? 16.0 : 8.0) * (double)triangles;
  *b_lists = !records  ? (double)hl + 60.0 * (double)triangles
             : in_place ? 48.0 * (double)triangles + 76.0 * (double)g.m
                        : 56.0 * (double)triangles + 56.0 * (double)g.m;
  return TRUSS_OK;
}

}  // namespace tr
