// Internal host-side interfaces between the translation units of the truss
// library.  Nothing here crosses the C ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "common.cuh"

namespace tr {

// Kernels launched by the calling host thread since the last reset (own
// kernels counted at each launch site, CUB calls by their pass count).
void count_launches(int k);
int64_t take_launches();

// Device workspace: a list of cudaMalloc'd chunks handed out by bump
// allocation.  reset() makes every chunk reusable without freeing it, so a
// steady stream of calls of similar size allocates nothing after the first.
// A call that needed more than one chunk leaves them folded into a single
// chunk of that call's peak size at the next reset(): chunks cut to one
// call's sizes fragment under a call that allocates in another order (a
// host-buffer call stages its inputs first), and near full device memory
// that fragmentation fails allocations that fit.
class Arena {
 public:
  ~Arena();
  void reset();
  // 256-byte aligned block, or nullptr if the device is out of memory.
  void *alloc(size_t bytes);
  template <class T>
  T *get(int64_t count) {
    return static_cast<T *>(alloc(sizeof(T) * (size_t)(count > 0 ? count : 1)));
  }
  size_t reserved() const;
  size_t unused() const;  // bytes of reserved chunks not handed out since reset()
  size_t peak() const { return peak_; }  // most bytes handed out at once since reset()
  // Cap on the bytes handed out since reset() (0 = none): alloc() returns
  // nullptr rather than exceed it.
  void set_limit(size_t bytes) { limit_ = bytes; }
  // Bytes alloc() can still hand out, given `free_dev` bytes of free device
  // memory: what the cap leaves, and no more than the reserved chunks' spare
  // room plus free_dev.
  size_t headroom(size_t free_dev) const;
  void release_all();
  // Allocation state, to hand back everything allocated after it (rewind);
  // chunks reserved since stay reserved.
  std::vector<size_t> mark() const;
  void rewind(const std::vector<size_t> &m);

 private:
  struct Chunk {
    char *p;
    size_t cap, used;
  };
  std::vector<Chunk> chunks_;
  size_t limit_ = 0;
  size_t handed_ = 0;  // bytes handed out since reset()
  size_t peak_ = 0;    // most bytes handed out at once since reset()
};

// ------------------------------------------------------------ CUB glue ---
// Thin wrappers around CUB's device-wide radix sort / scan (cub_ops.cu).
// `tmp` == nullptr queries the scratch size into *tmp_bytes.
int sort_pairs_u64(void *tmp, size_t *tmp_bytes, const uint64_t *kin, uint64_t *kout,
                   const int32_t *vin, int32_t *vout, int64_t n, int begin_bit, int end_bit,
                   cudaStream_t s);
int sort_keys_u64(void *tmp, size_t *tmp_bytes, const uint64_t *kin, uint64_t *kout, int64_t n,
                  int begin_bit, int end_bit, cudaStream_t s);
int sort_pairs_u32(void *tmp, size_t *tmp_bytes, const uint32_t *kin, uint32_t *kout,
                   const int32_t *vin, int32_t *vout, int64_t n, int begin_bit, int end_bit,
                   cudaStream_t s);
int inclusive_sum_i32(void *tmp, size_t *tmp_bytes, const int32_t *in, int32_t *out, int64_t n,
                      cudaStream_t s);
int exclusive_sum_i64(void *tmp, size_t *tmp_bytes, const int64_t *in, int64_t *out, int64_t n,
                      cudaStream_t s);

// ---------------------------------------------------------- CSR build ---
// Input rows as seen by the device (already staged into device memory).
struct RowsIn {
  int64_t rows = 0;
  int64_t n = 0;                 // total vertex count (sum over graphs for a batch)
  const int32_t *src = nullptr;  // device
  const int32_t *dst = nullptr;  // device
  // batch: G graphs, device arrays row_off[G+1], voff[G+1] (vertex offsets)
  int32_t graphs = 1;
  const int64_t *row_off = nullptr;
  const int64_t *voff = nullptr;
};

// Degree-ordered oriented CSR (vertices relabelled by ascending (degree, id)
// so that an edge points from its lower-ranked to its higher-ranked end).
// Canonical edge id e = position in adjp.
struct Csr {
  int64_t n = 0, m = 0, rows = 0;
  int64_t *offp = nullptr;   // [n+1] out-list offsets (new labels)
  int32_t *adjp = nullptr;   // [m]   head (higher-ranked endpoint) of edge e
  int32_t *esrc = nullptr;   // [m]   tail (lower-ranked endpoint) of edge e
  int32_t *row2e = nullptr;  // [rows] row -> e, -1 for self-loop rows
  int32_t *order = nullptr;  // [n]   rank -> input vertex id
};

struct DevCounters;  // device scratch for small counters (api.cu)

int build_csr(Arena &A, const RowsIn &in, Csr *out, int32_t *d_err, cudaStream_t s);

// ------------------------------------------------------------- support ---
struct SupportOut {
  int32_t *sup = nullptr;    // [m]  sup(e)
  int32_t *supA = nullptr;   // [m]  triangles in which e is e_uv or e_uw (e in out(u))
  int64_t *toff = nullptr;   // [m+1] triangle-list offsets (exclusive sum of sup)
  int64_t walk = 0;          // total walk cost (out-list entries probed, plus fixed costs)
  int32_t *inedge = nullptr; // [m]  edges grouped by head
  int64_t *inoff = nullptr;  // [n+1] start of each head's group in inedge
  int64_t entries = 0;       // sum sup = 3 * triangles
  // optional triangle records of the support walk (see support.cu)
  int64_t *tbpre = nullptr;  // [m+1] record-region offsets
  int64_t records = 0;       // size of the record regions (record indices are below it)
  int2 *tb = nullptr;        // (e_uw, e_vw) records per walked edge e_uv
  int32_t *cuv = nullptr;    // [m] records per edge
  bool in_place = false;     // the lists keep each edge's own part in its records
};

struct SupportCfg {
  int block = 256;
  int sms = 0;
  bool records = false;  // also record triangles for the list pass (if memory allows)
  bool full_lists = false;  // the lists must be whole (the barrier-free peel's layout)
  bool in_place = false;    // own parts in place whenever records are used
  int pair_cost = 0;      // fixed cost per oriented edge, in out-list entries (0 = default, <0 = none)
  int64_t range_work = 0; // walk cost per range (0 = default)
  int stage_max = 0;      // stage out-lists of at most this many entries (0 = capacity)
};

// Support of every edge: sup = supA + supB (support.cu).
int run_support(Arena &A, const Csr &g, const SupportCfg &cfg, SupportOut *out, cudaStream_t s);
// Where the triangle list of each edge lives: for edge e, the other two
// edge ids of each triangle of e are own[own_off[e] .. own_off[e] +
// own_cnt[e]) followed by rest[off[e] .. off[e] + sup[e] - own_cnt[e]).
// With the own parts in place (SupportOut::in_place), the own part is e's
// records (the triangles e closes as the walked edge), left where the support
// walk wrote them, and rest holds only the two partner copies of each
// triangle; otherwise own_cnt is null and rest[toff[e] ..) holds e's whole
// list.
struct TriLists {
  const int2 *own = nullptr;
  const int64_t *own_off = nullptr;
  const int32_t *own_cnt = nullptr;
  const int2 *rest = nullptr;
  const int64_t *off = nullptr;
};

// Entries the lists' `rest` array needs: 2T with the own parts in place,
// else all 3T.
inline int64_t list_rest_entries(const SupportOut &so) {
  return (so.tb && so.in_place) ? so.entries - so.entries / 3 : so.entries;
}

// Triangle lists (support.cu) into `pairs` (list_rest_entries entries).
// tids (nullable, only with records and whole lists): the record index of
// each entry's triangle, for the barrier-free peel.
int run_lists(Arena &A, const Csr &g, const SupportCfg &cfg, const SupportOut &so, int2 *pairs,
              uint32_t *tids, TriLists *out, cudaStream_t s);

// ---------------------------------------------------------------- peel ---
struct PeelCfg {
  int block = 512;
  int variant = 0;  // kernel shape (peel.cu: run_peel)
  int sms = 0;
  long long wait_ns = 4000000000LL;
  // Optional: edges never removed (their triangles still count), and the
  // last level to run (0 = all).  Edges not removed by then get truss 0.
  const uint8_t *pinned = nullptr;
  int k_stop = 0;
  // Counting run (untimed): record each edge's removal sub-round and the
  // per-level list-entry counts, and compute the algorithmic bytes of the
  // removals (PeelResult::sum_min_alive .. alive_levels).
  bool count = false;
};

struct PeelResult {
  int32_t kmax = 0, levels = 0, subrounds = 0, err = 0;
  unsigned long long entries = 0, decrements = 0, scanned = 0;
  // counting runs only:
  //  sum_min_alive = sum over edges e = (u, v) of min(L_u, L_v), L_x = 1 +
  //    the number of x's edges removed in a later sub-round than e (e last
  //    among the edges its sub-round removes); sum_min_alive_start counts
  //    in L_x every edge of x not removed before e's sub-round;
  //  alive_levels = sum over the levels k that remove an edge of the edges
  //    present when level k starts;
  //  dead = list entries read whose triangle had already lost an edge,
  //    dead_earlier = those whose triangle lost it in an earlier level.
  unsigned long long sum_min_alive = 0, sum_min_alive_start = 0, alive_levels = 0, dead = 0,
                     dead_earlier = 0;
};

// Barrier-free peel (peel_async.cu): needs the list entries' triangle ids
// (record indices below ntri).
int run_peel_async(Arena &A, const Csr &g, const SupportOut &so, const int2 *pairs,
                   const uint32_t *tids, int64_t ntri, const PeelCfg &cfg, int32_t *truss,
                   PeelResult *out, cudaStream_t s);
int run_peel(Arena &A, const Csr &g, const SupportOut &so, const TriLists &L, const PeelCfg &cfg,
             int32_t *truss, PeelResult *res, cudaStream_t s);
// sum[0] = sum_min_alive, sum[1] = sum_min_alive_start (see PeelResult) from
// each edge's removal sub-round `when` (peel.cu).
int count_min_alive(Arena &A, const Csr &g, const SupportOut &so, const int32_t *when,
                    unsigned long long *sum, cudaStream_t s);

// -------------------------------------------------------------- outputs ---
int scatter_rows(const Csr &g, const int32_t *sup, const int32_t *truss, int32_t *sup_rows,
                 int32_t *truss_rows, cudaStream_t s);
// The same through a packed (support, truss) pair per edge when both outputs
// are wanted and the workspace has room for it.
int scatter_rows_packed(Arena &A, const Csr &g, const int32_t *sup, const int32_t *truss,
                        int32_t *sup_rows, int32_t *truss_rows, cudaStream_t s);
int batch_kmax(int32_t G, const int64_t *row_off, const int32_t *truss_rows, int32_t *kmax,
               cudaStream_t s);
// Per-graph distinct edges and support sums of a batch (voff: device vertex
// offsets, G+1 entries); results are added into m_g and sup_g (device, G).
int batch_graph_counts(const Csr &g, int32_t G, const int64_t *voff, const int32_t *sup,
                       unsigned long long *m_g, unsigned long long *sup_g, cudaStream_t s);

// Algorithmic byte counts (see the comments in support.cu / peel.cu).
// ------------------------------------------------------------ top-t ---
// psi(e) = min{sup(e), x_u, x_v} + 2 of every edge (Procedure 6 with the
// whole graph as H) (topt.cu).
int compute_psi(Arena &A, const Csr &g, const int32_t *sup, int32_t *psi, cudaStream_t s);
// Largest psi and the count of edges with psi >= k for k = 0 .. max psi
// (host vector, cnt_ge[k]).
int psi_counts(Arena &A, int64_t m, const int32_t *psi, std::vector<int64_t> *cnt_ge,
               cudaStream_t s);
// Edges with psi >= k_lo as rows (u, v) of the relabelled graph and their edge
// ids; *mc receives their number.
int select_candidates(Arena &A, const Csr &g, const int32_t *psi, int32_t k_lo, int32_t *cs,
                      int32_t *cd, int32_t *ce, int64_t *mc, cudaStream_t s);
// top[e] = phi_rows[r] for candidate r with e = ce[r] if phi_rows[r] >= thr,
// every other entry 0.
int top_classes(int64_t m, int64_t mc, const int32_t *ce, const int32_t *phi_rows, int32_t thr,
                int32_t *top, cudaStream_t s);

// ---------------------------------------------------- bottom-up (budget) ---
// Helpers of the budgeted bottom-up decomposition (bottomup.cu); edge state
// 0 = in G (Algorithm 3), 1 = in G_new, 2 = truss number known.
int bu_list_state(Arena &A, int64_t m, const uint8_t *state, int want, int32_t *out,
                  int64_t *count, cudaStream_t s);
int bu_degrees(int64_t n, int64_t nl, const int32_t *list, const int32_t *eu, const int32_t *ev,
               int32_t *deg, cudaStream_t s);
int bu_select_range(Arena &A, int64_t nl, const int32_t *list, const int32_t *eu,
                    const int32_t *ev, int32_t va, int32_t vb, int32_t *hs, int32_t *hd,
                    int32_t *hid, int64_t *mh, cudaStream_t s);
int bu_alg3_update(int64_t mh, const int32_t *hid, const int32_t *hs, const int32_t *hd,
                   int32_t va, int32_t vb, const int32_t *truss_h, int32_t *lower, int32_t *phi,
                   uint8_t *state, cudaStream_t s);
int bu_min_lower(Arena &A, int64_t nl, const int32_t *list, const int32_t *lower, int32_t *mn,
                 cudaStream_t s);
int bu_select_candidates(Arena &A, int64_t n, int64_t nl, const int32_t *list, const int32_t *eu,
                         const int32_t *ev, const int32_t *lower, int32_t k, uint8_t *inU,
                         int32_t *hs, int32_t *hd, int32_t *hid, uint8_t *pinned, int64_t *mh,
                         cudaStream_t s);
int bu_assign(int64_t mh, const int32_t *hid, const uint8_t *pinned, const int32_t *truss_h,
              int32_t k, int32_t *phi, uint8_t *state, cudaStream_t s);
int bu_max(Arena &A, int64_t m, const int32_t *x, int32_t *mx, cudaStream_t s);
// pinned_e[row2e[r]] = 1 for rows with pinned_rows[r] (others 0).
int pin_edges(int64_t rows, const int32_t *row2e, const uint8_t *pinned_rows, uint8_t *pinned_e,
              int64_t m, cudaStream_t s);

// ------------------------------------------------------------- k-core ---
// Core number of every vertex, written to core_out[input vertex id] (core.cu).
int run_core(Arena &A, const Csr &g, int sms, long long wait_ns, int32_t *core_out,
             int32_t *kmax, int32_t *levels, int32_t *subrounds, cudaStream_t s);

// Algorithmic bytes of the support pass: b_sup by the per-edge formula
// 4 * sum over oriented edges (u, v) of (d+(u) + d+(v)) + 44 m + 24 T (a
// forward merge of the two out-lists of every edge, its offsets, endpoints,
// support write and the three read-modify-writes per triangle); b_sup_design
// by the per-unit figures of the walk this library runs (support.cu); b_lists
// of the list passes.
int count_support_bytes(Arena &A, const Csr &g, int64_t triangles, bool records, bool in_place,
                        double *b_sup, double *b_sup_design, double *b_lists, cudaStream_t s);

}  // namespace tr
