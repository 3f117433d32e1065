// C ABI of the truss library (include/truss.h): contexts, argument checks,
// host/device staging, and the single-graph / batched pipelines.
//
// Pipeline of one call (all kernels on the caller's stream):
//   build_csr   rows -> degree-ordered oriented CSR, row -> edge id
//   run_support sup(e) (Definition 1, Algorithm 2 step 2)
//   run_lists   per-edge triangle lists (edge-id pairs)
//   run_peel    truss numbers (Algorithm 2 steps 3-16), one persistent launch
//   scatter     per-row outputs
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "engine.h"

struct truss_ctx {
  int device = 0;
  truss_opts opts{};
  tr::Arena arena;
  int32_t *d_err = nullptr;  // device error word for argument checks
  truss_run_stats last{};
  cudaEvent_t ev[8] = {};
  bool have_events = false;
  int sms = 0;
};

namespace tr {

namespace {
thread_local std::string g_last_cuda_error;
thread_local int64_t g_launches = 0;
}

void count_launches(int k) { g_launches += k; }
int64_t take_launches() {
  int64_t v = g_launches;
  g_launches = 0;
  return v;
}

void note_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_cuda_error = buf;
  if (getenv("TRUSS_VERBOSE")) fprintf(stderr, "[truss] %s\n", buf);
}

// ------------------------------------------------------------------ Arena ---
Arena::~Arena() { release_all(); }

void Arena::release_all() {
  for (auto &c : chunks_) cudaFree(c.p);
  chunks_.clear();
  handed_ = 0;
  peak_ = 0;
}

void Arena::reset() {
  size_t live = 0;
  for (auto &c : chunks_) live += c.cap > 0;
  if (live > 1 && peak_ > 0) {
    const size_t want = peak_;
    release_all();
    char *p = nullptr;
    if (cudaMalloc(&p, want) == cudaSuccess) {
      chunks_.push_back(Chunk{p, want, 0});
    } else {
      cudaGetLastError();  // leave it to alloc() to grow again
    }
  }
  for (auto &c : chunks_) c.used = 0;
  handed_ = 0;
  peak_ = 0;
}

size_t Arena::headroom(size_t free_dev) const {
  const size_t room = unused() + free_dev;
  if (!limit_) return room;
  const size_t left = limit_ > handed_ ? limit_ - handed_ : 0;
  return left < room ? left : room;
}

size_t Arena::unused() const {
  size_t s = 0;
  for (auto &c : chunks_) s += c.cap - c.used;
  return s;
}

size_t Arena::reserved() const {
  size_t s = 0;
  for (auto &c : chunks_) s += c.cap;
  return s;
}

std::vector<size_t> Arena::mark() const {
  std::vector<size_t> m;
  for (auto &c : chunks_) m.push_back(c.used);
  return m;
}

void Arena::rewind(const std::vector<size_t> &m) {
  handed_ = 0;
  for (size_t i = 0; i < chunks_.size(); i++) {
    chunks_[i].used = i < m.size() ? m[i] : 0;
    handed_ += chunks_[i].used;
  }
}

void *Arena::alloc(size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  if (limit_ && handed_ + bytes > limit_) return nullptr;
  for (auto &c : chunks_) {
    if (c.cap - c.used >= bytes) {
      void *p = c.p + c.used;
      c.used += bytes;
      handed_ += bytes;
      if (handed_ > peak_) peak_ = handed_;
      return p;
    }
  }
  size_t cap = bytes < ((size_t)64 << 20) ? ((size_t)64 << 20) : bytes;
  char *p = nullptr;
  if (cudaMalloc(&p, cap) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free allocation error
    // Chunks are cut to the sizes an earlier call asked for; a call that
    // allocates in another order may find none that fits while most of them
    // are still untouched since reset().  Give those back and retry once.
    // They stay in the list as empty entries, so the chunk indices that
    // mark() records keep their meaning.
    bool freed = false;
    for (auto &c : chunks_) {
      if (c.used == 0 && c.cap > 0) {
        cudaFree(c.p);
        c.p = nullptr;
        c.cap = 0;
        freed = true;
      }
    }
    if (!freed || cudaMalloc(&p, cap) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  chunks_.push_back(Chunk{p, cap, bytes});
  handed_ += bytes;
  if (handed_ > peak_) peak_ = handed_;
  return p;
}

// ------------------------------------------------------------ scatter ---
namespace {
__global__ void k_scatter(int64_t rows, const int32_t *row2e, const int32_t *sup,
                          const int32_t *truss, int32_t *sup_rows, int32_t *truss_rows) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = row2e[r];
    if (sup_rows) sup_rows[r] = e < 0 ? -1 : sup[e];
    if (truss_rows) truss_rows[r] = e < 0 ? -1 : truss[e];
  }
}

// Support and truss number of each edge side by side, so that the per-row
// scatter gathers one 8-byte pair per row instead of two scattered words.
__global__ void k_pack(int64_t m, const int32_t *sup, const int32_t *truss, int2 *pk) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    pk[e] = make_int2(sup[e], truss[e]);
}

__global__ void k_scatter_pk(int64_t rows, const int32_t *row2e, const int2 *pk,
                             int32_t *sup_rows, int32_t *truss_rows) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = row2e[r];
    const int2 v = e < 0 ? make_int2(-1, -1) : pk[e];
    sup_rows[r] = v.x;
    truss_rows[r] = v.y;
  }
}

// One block per graph: k_max = max truss number over its rows.
__global__ void k_batch_kmax(int32_t G, const int64_t *row_off, const int32_t *truss_rows,
                             int32_t *kmax) {
  __shared__ int red[32];
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    int best = 0;
    for (int64_t r = row_off[g] + threadIdx.x; r < row_off[g + 1]; r += blockDim.x)
      best = max(best, truss_rows[r]);
    best = __reduce_max_sync(TR_FULL, best);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
      int v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
      v = __reduce_max_sync(TR_FULL, v);
      if (threadIdx.x == 0) kmax[g] = v;
    }
    __syncthreads();
  }
}
// Graph of each canonical edge (from its tail's input id) -> per-graph
// distinct edges and support sums.
__global__ void k_graph_counts(int64_t m, int32_t G, const int64_t *voff, const int32_t *order,
                               const int32_t *esrc, const int32_t *sup, unsigned long long *m_g,
                               unsigned long long *sup_g) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = order[esrc[e]];
    int lo = 0, hi = G - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (voff[mid] <= x) lo = mid; else hi = mid - 1;
    }
    atomicAdd(&m_g[lo], 1ull);
    atomicAdd(&sup_g[lo], (unsigned long long)sup[e]);
  }
}
}  // namespace

int batch_graph_counts(const Csr &g, int32_t G, const int64_t *voff, const int32_t *sup,
                       unsigned long long *m_g, unsigned long long *sup_g, cudaStream_t s) {
  if (g.m == 0 || G <= 0) return TRUSS_OK;
  k_graph_counts<<<grid_for(g.m, 256, 152 * 16), 256, 0, s>>>(g.m, G, voff, g.order, g.esrc, sup,
                                                              m_g, sup_g);
  TR_LAUNCHED();
  return TRUSS_OK;
}

int scatter_rows(const Csr &g, const int32_t *sup, const int32_t *truss, int32_t *sup_rows,
                 int32_t *truss_rows, cudaStream_t s) {
  if (g.rows == 0) return TRUSS_OK;
  k_scatter<<<grid_for(g.rows, 256, 152 * 16), 256, 0, s>>>(g.rows, g.row2e, sup, truss, sup_rows,
                                                             truss_rows);
  TR_LAUNCHED();
  return TRUSS_OK;
}

int scatter_rows_packed(Arena &A, const Csr &g, const int32_t *sup, const int32_t *truss,
                        int32_t *sup_rows, int32_t *truss_rows, cudaStream_t s) {
  int2 *pk = (sup_rows && truss_rows && g.m > 0) ? A.get<int2>(g.m) : nullptr;
  if (!pk) return scatter_rows(g, sup, truss, sup_rows, truss_rows, s);
  k_pack<<<grid_for(g.m, 256, 152 * 16), 256, 0, s>>>(g.m, sup, truss, pk);
  TR_LAUNCHED();
  k_scatter_pk<<<grid_for(g.rows, 256, 152 * 16), 256, 0, s>>>(g.rows, g.row2e, pk, sup_rows,
                                                                truss_rows);
  TR_LAUNCHED();
  return TRUSS_OK;
}

int batch_kmax(int32_t G, const int64_t *row_off, const int32_t *truss_rows, int32_t *kmax,
               cudaStream_t s) {
  if (G <= 0) return TRUSS_OK;
  k_batch_kmax<<<G < 4096 ? G : 4096, 256, 0, s>>>(G, row_off, truss_rows, kmax);
  TR_LAUNCHED();
  return TRUSS_OK;
}

}  // namespace tr

// ================================================================== C ABI ===
namespace {

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device address of pinned (page-locked) host memory, or nullptr for any
// other memory.  Kernels can read and write pinned memory in place over the
// host link (NVLink-C2C on Grace machines), which moves each byte once and
// needs no staging buffer.
void *pinned_view(const void *p) {
  cudaPointerAttributes at{};
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Device-usable input: device memory as is; with `direct`, pinned host
// memory in place (for inputs one kernel reads once); otherwise a staged
// copy in the arena.
template <class T>
int stage_in(tr::Arena &A, const T *p, int64_t count, const T **out, cudaStream_t s,
             bool direct = false) {
  if (count == 0 || p == nullptr || is_device_ptr(p)) {
    *out = p;
    return TRUSS_OK;
  }
  if (direct) {
    if (const void *dp = pinned_view(p)) {
      *out = (const T *)dp;
      return TRUSS_OK;
    }
  }
  T *d = A.get<T>(count);
  if (!d) return TRUSS_ENOMEM;
  TR_CUDA(cudaMemcpyAsync(d, p, sizeof(T) * count, cudaMemcpyHostToDevice, s));
  *out = d;
  return TRUSS_OK;
}

struct OutBuf {
  int32_t *user = nullptr;
  int32_t *dev = nullptr;
  bool host = false;
};

// Device-usable output: device memory as is; with `direct`, pinned host
// memory written in place; otherwise an arena buffer copied back.
int stage_out(tr::Arena &A, int32_t *user, int64_t count, OutBuf *o, bool direct = false) {
  o->user = user;
  o->host = false;
  o->dev = user;
  if (!user) return TRUSS_OK;
  if (!is_device_ptr(user)) {
    if (direct) {
      if (void *dp = pinned_view(user)) {
        o->dev = (int32_t *)dp;
        return TRUSS_OK;
      }
    }
    o->host = true;
    o->dev = A.get<int32_t>(count);
    if (!o->dev) return TRUSS_ENOMEM;
  }
  return TRUSS_OK;
}

int copy_back(const OutBuf &o, int64_t count, cudaStream_t s) {
  if (o.user && o.host && count > 0)
    TR_CUDA(cudaMemcpyAsync(o.user, o.dev, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s));
  return TRUSS_OK;
}

struct Stage {
  truss_ctx *c;
  cudaStream_t s;
  int next = 0;
  void mark() {
    if (c->opts.profile && c->have_events && next < 8) cudaEventRecord(c->ev[next++], s);
  }
  float ms(int a, int b) const {
    float t = 0.f;
    if (b < next && a < b) cudaEventElapsedTime(&t, c->ev[a], c->ev[b]);
    return t;
  }
};

int run_pipeline(truss_ctx *ctx, int64_t n_total, int64_t rows, const int32_t *src,
                 const int32_t *dst, int32_t G, const int64_t *h_row_off, const int64_t *h_voff,
                 int32_t *support_out, int32_t *truss_out, int32_t *kmax_out, bool want_truss,
                 cudaStream_t s, int64_t *graph_m = nullptr, int64_t *graph_tri = nullptr) {
  TR_CUDA(cudaSetDevice(ctx->device));
  tr::Arena &A = ctx->arena;
  A.reset();
  tr::take_launches();
  truss_run_stats st{};
  st.n = n_total;
  st.rows = rows;
  st.graphs = G;
  Stage sg{ctx, s};
  sg.mark();  // 0

  tr::RowsIn in;
  in.rows = rows;
  in.n = n_total;
  // the rows are read once, by the key kernel: pinned host rows in place
  TR_TRY(stage_in(A, src, rows, &in.src, s, true));
  TR_TRY(stage_in(A, dst, rows, &in.dst, s, true));
  int64_t *d_row_off = nullptr, *d_voff = nullptr;
  if (h_row_off) {
    d_row_off = A.get<int64_t>(G + 1);
    d_voff = A.get<int64_t>(G + 1);
    if (!d_row_off || !d_voff) return TRUSS_ENOMEM;
    TR_CUDA(cudaMemcpyAsync(d_row_off, h_row_off, sizeof(int64_t) * (G + 1),
                            cudaMemcpyHostToDevice, s));
    TR_CUDA(cudaMemcpyAsync(d_voff, h_voff, sizeof(int64_t) * (G + 1), cudaMemcpyHostToDevice,
                            s));
    in.graphs = G;
    in.row_off = d_row_off;
    in.voff = d_voff;
  }
  TR_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), s));

  tr::Csr g;
  TR_TRY(tr::build_csr(A, in, &g, ctx->d_err, s));
  sg.mark();  // 1
  st.m = g.m;

  tr::SupportCfg scfg;
  scfg.sms = ctx->sms;
  scfg.records = want_truss && !ctx->opts.lists_by_walk;
  scfg.full_lists = ctx->opts.peel_variant == 4;
  scfg.in_place = ctx->opts.lists_in_place != 0;
  scfg.pair_cost = ctx->opts.support_pair_cost;
  scfg.range_work = ctx->opts.support_range_work;
  scfg.stage_max = ctx->opts.support_stage_max;
  tr::SupportOut so;
  TR_TRY(tr::run_support(A, g, scfg, &so, s));
  sg.mark();  // 2
  st.triangles = so.entries / 3;
  if (graph_m && h_row_off) {
    unsigned long long *cnt = A.get<unsigned long long>(2 * (int64_t)G);
    if (!cnt) return TRUSS_ENOMEM;
    TR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 2 * G, s));
    TR_TRY(tr::batch_graph_counts(g, G, d_voff, so.sup, cnt, cnt + G, s));
    std::vector<unsigned long long> h((size_t)2 * G);
    TR_CUDA(cudaMemcpyAsync(h.data(), cnt, sizeof(unsigned long long) * 2 * G,
                            cudaMemcpyDeviceToHost, s));
    TR_CUDA(cudaStreamSynchronize(s));
    for (int32_t i = 0; i < G; i++) {
      graph_m[i] = (int64_t)h[i];
      graph_tri[i] = (int64_t)(h[G + i] / 3);
    }
  }

  int32_t *truss_e = nullptr;
  tr::PeelResult pr;
  if (want_truss) {
    // peel variant 4: the barrier-free peel, which needs the full lists and
    // a triangle id per list entry (record indices, so records and fewer
    // than 2^32 of them)
    const bool async = ctx->opts.peel_variant == 4 && so.tb && !so.in_place &&
                       so.records < ((int64_t)1 << 32);
    int2 *pairs = A.get<int2>(tr::list_rest_entries(so));
    truss_e = A.get<int32_t>(g.m);
    if (!pairs || !truss_e) return TRUSS_ENOMEM;
    // short of memory for the ids, the full lists go to the level-synchronous peel
    uint32_t *tids = async ? A.get<uint32_t>(so.entries) : nullptr;
    tr::TriLists lists;
    TR_TRY(tr::run_lists(A, g, scfg, so, pairs, tids, &lists, s));
    st.lists_layout = !so.tb ? 1 : so.in_place ? 3 : 2;
    sg.mark();  // 3
    tr::PeelCfg pcfg;
    pcfg.sms = ctx->sms;
    pcfg.variant = ctx->opts.peel_variant;
    pcfg.count = ctx->opts.count_bytes != 0 && !tids;
    if (ctx->opts.wait_limit_ns > 0) pcfg.wait_ns = ctx->opts.wait_limit_ns;
    int rc = tids ? tr::run_peel_async(A, g, so, pairs, tids, so.records, pcfg, truss_e, &pr, s)
                  : tr::run_peel(A, g, so, lists, pcfg, truss_e, &pr, s);
    if (rc != TRUSS_OK) return rc;
    sg.mark();  // 4
    st.kmax = pr.kmax;
    st.levels = pr.levels;
    st.subrounds = pr.subrounds;
    st.peel_entries = (int64_t)pr.entries;
    st.peel_decrements = (int64_t)pr.decrements;
    st.peel_scanned = (int64_t)pr.scanned;
  }

  // the per-row outputs are written once, by the scatter: pinned host
  // outputs in place
  OutBuf os, ot;
  TR_TRY(stage_out(A, support_out, rows, &os, true));
  TR_TRY(stage_out(A, want_truss ? truss_out : nullptr, rows, &ot, true));
  TR_TRY(tr::scatter_rows_packed(A, g, so.sup, truss_e, os.dev, ot.dev, s));
  if (G > 1 || h_row_off) {
    if (kmax_out && want_truss) {
      OutBuf ok;
      TR_TRY(stage_out(A, kmax_out, G, &ok));
      TR_TRY(tr::batch_kmax(G, d_row_off, ot.dev, ok.dev, s));
      TR_TRY(copy_back(ok, G, s));
    }
  }
  TR_TRY(copy_back(os, rows, s));
  TR_TRY(copy_back(ot, rows, s));
  sg.mark();  // 5 (or 3 for support only)
  int32_t k_host = pr.kmax;
  if (!(G > 1 || h_row_off) && kmax_out && want_truss) {
    if (is_device_ptr(kmax_out)) {
      TR_CUDA(cudaMemcpyAsync(kmax_out, &k_host, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    } else {
      *kmax_out = k_host;
    }
  }
  TR_CUDA(cudaStreamSynchronize(s));
  if (ctx->opts.profile && ctx->have_events) {
    st.ms_build = sg.ms(0, 1);
    st.ms_support = sg.ms(1, 2);
    if (want_truss) {
      st.ms_lists = sg.ms(2, 3);
      st.ms_peel = sg.ms(3, 4);
      st.ms_scatter = sg.ms(4, 5);
      st.ms_total = sg.ms(0, 5);
    } else {
      st.ms_scatter = sg.ms(2, 3);
      st.ms_total = sg.ms(0, 3);
    }
  }
  st.launches = tr::take_launches();
  st.workspace_bytes = (int64_t)A.reserved();
  st.workspace_peak = (int64_t)A.peak();
  if (ctx->opts.count_bytes) {
    double bs = 0, bsd = 0, bl = 0;
    TR_TRY(tr::count_support_bytes(A, g, st.triangles, so.tb != nullptr, so.in_place, &bs, &bsd,
                                   &bl, s));
    st.bytes_support = bs;
    st.design_bytes_support = bsd;
    st.bytes_lists = want_truss ? bl : 0.0;
    if (want_truss) {
      st.design_bytes_peel = (so.in_place ? 40.0 : 28.0) * (double)g.m +
                             16.0 * (double)pr.entries + 8.0 * (double)pr.decrements +
                             16.0 * (double)pr.scanned;
      const double smin = (double)pr.sum_min_alive;
      st.bytes_peel = 12.0 * smin + 12.0 * (smin - (double)g.m) + 8.0 * (double)g.m +
                      16.0 * (double)st.triangles + 8.0 * (double)pr.alive_levels;
      st.peel_sum_min_alive = (int64_t)pr.sum_min_alive;
      st.peel_sum_min_alive_start = (int64_t)pr.sum_min_alive_start;
      st.peel_alive_levels = (int64_t)pr.alive_levels;
      st.peel_dead_entries = (int64_t)pr.dead;
      st.peel_dead_earlier = (int64_t)pr.dead_earlier;
    }
  }
  ctx->last = st;
  return TRUSS_OK;
}

int check_common(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src, const int32_t *dst) {
  if (!ctx) return TRUSS_EINVAL;
  if (n < 0 || n >= ((int64_t)1 << 31)) return TRUSS_EINVAL;
  if (rows < 0 || rows >= ((int64_t)1 << 31)) return TRUSS_EINVAL;
  if (rows > 0 && (!src || !dst)) return TRUSS_EINVAL;
  if (rows > 0 && n == 0) return TRUSS_EINVAL;
  return TRUSS_OK;
}

// The whole pipeline (CSR build, support, lists, peel) on rows already in
// device memory: per-row support (nullable) and truss number.  Optional:
// rows whose edges are never removed (pinned_rows) and the last level to run
// (k_stop); edges not removed by then get truss 0.
int decompose_device_rows(truss_ctx *ctx, tr::Arena &A, const tr::RowsIn &in, int32_t *sup_rows,
                          int32_t *truss_rows, const uint8_t *pinned_rows, int32_t k_stop,
                          tr::PeelResult *pr, cudaStream_t s) {
  *pr = tr::PeelResult{};
  if (in.rows == 0) return TRUSS_OK;
  tr::Csr g;
  TR_TRY(tr::build_csr(A, in, &g, ctx->d_err, s));
  tr::SupportCfg cfg;
  cfg.sms = ctx->sms;
  cfg.records = true;
  cfg.in_place = ctx->opts.lists_in_place != 0;
  cfg.pair_cost = ctx->opts.support_pair_cost;
  cfg.range_work = ctx->opts.support_range_work;
  cfg.stage_max = ctx->opts.support_stage_max;
  tr::SupportOut so;
  TR_TRY(tr::run_support(A, g, cfg, &so, s));
  int2 *pairs = A.get<int2>(tr::list_rest_entries(so));
  int32_t *truss_e = A.get<int32_t>(g.m);
  if (!pairs || !truss_e) return TRUSS_ENOMEM;
  tr::TriLists lists;
  TR_TRY(tr::run_lists(A, g, cfg, so, pairs, nullptr, &lists, s));
  tr::PeelCfg pcfg;
  pcfg.sms = ctx->sms;
  pcfg.variant = ctx->opts.peel_variant;
  if (ctx->opts.wait_limit_ns > 0) pcfg.wait_ns = ctx->opts.wait_limit_ns;
  pcfg.k_stop = k_stop;
  if (pinned_rows) {
    uint8_t *pe = A.get<uint8_t>(g.m);
    if (!pe) return TRUSS_ENOMEM;
    TR_TRY(tr::pin_edges(g.rows, g.row2e, pinned_rows, pe, g.m, s));
    pcfg.pinned = pe;
  }
  int rc = tr::run_peel(A, g, so, lists, pcfg, truss_e, pr, s);
  if (rc != TRUSS_OK) return rc;
  return tr::scatter_rows(g, so.sup, truss_e, sup_rows, truss_rows, s);
}

// Per-row support and psi (Procedure 6) of the graph the rows define.
int run_upper_bound(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src,
                    const int32_t *dst, int32_t *support_out, int32_t *psi_out, cudaStream_t s) {
  TR_CUDA(cudaSetDevice(ctx->device));
  tr::Arena &A = ctx->arena;
  A.reset();
  tr::take_launches();
  truss_run_stats st{};
  st.n = n;
  st.rows = rows;
  st.graphs = 1;
  tr::RowsIn in;
  in.rows = rows;
  in.n = n;
  TR_TRY(stage_in(A, src, rows, &in.src, s));
  TR_TRY(stage_in(A, dst, rows, &in.dst, s));
  TR_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), s));
  tr::Csr g;
  TR_TRY(tr::build_csr(A, in, &g, ctx->d_err, s));
  st.m = g.m;
  tr::SupportCfg scfg;
  scfg.sms = ctx->sms;
  scfg.pair_cost = ctx->opts.support_pair_cost;
  scfg.range_work = ctx->opts.support_range_work;
  scfg.stage_max = ctx->opts.support_stage_max;
  tr::SupportOut so;
  TR_TRY(tr::run_support(A, g, scfg, &so, s));
  st.triangles = so.entries / 3;
  int32_t *psi = A.get<int32_t>(g.m);
  if (!psi) return TRUSS_ENOMEM;
  TR_TRY(tr::compute_psi(A, g, so.sup, psi, s));
  OutBuf os, op;
  TR_TRY(stage_out(A, support_out, rows, &os));
  TR_TRY(stage_out(A, psi_out, rows, &op));
  TR_TRY(tr::scatter_rows(g, so.sup, psi, os.dev, op.dev, s));
  TR_TRY(copy_back(os, rows, s));
  TR_TRY(copy_back(op, rows, s));
  TR_CUDA(cudaStreamSynchronize(s));
  st.launches = tr::take_launches();
  ctx->last = st;
  return TRUSS_OK;
}

// Top-t classes (Algorithm 7): supports and psi of the whole graph, then the
// full pipeline on the candidate subgraph {e : psi(e) >= k_lo}, which gives
// every truss number >= k_lo exactly (Lemma 2).  k_lo starts at kb - t + 1,
// kb the largest k with at least k(k-1)/2 edges of psi >= k (a bound on
// k_max), and is lowered until k_lo <= k_max - t + 1:
//  * T_{k_lo} empty in the candidate (its k_max' < k_lo): k_max(G) lies in
//    [k_max', k_lo - 1] (a subgraph's k-trusses lie in the graph's), so
//    k_lo = k_max' - t + 1 is low enough and that round is the last;
//  * otherwise k_max = k_max' exactly, and one more round with
//    k_lo = k_max - t + 1 follows if needed.
// At most two rounds after the first.
int run_top(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
            int32_t t, int32_t *truss_out, int32_t *kmax_out, cudaStream_t s) {
  TR_CUDA(cudaSetDevice(ctx->device));
  tr::Arena &A = ctx->arena;
  A.reset();
  tr::take_launches();
  truss_run_stats st{};
  st.n = n;
  st.rows = rows;
  st.graphs = 1;
  Stage sg{ctx, s};
  sg.mark();  // 0
  tr::RowsIn in;
  in.rows = rows;
  in.n = n;
  TR_TRY(stage_in(A, src, rows, &in.src, s));
  TR_TRY(stage_in(A, dst, rows, &in.dst, s));
  TR_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), s));
  tr::Csr g;
  TR_TRY(tr::build_csr(A, in, &g, ctx->d_err, s));
  st.m = g.m;
  tr::SupportCfg scfg;
  scfg.sms = ctx->sms;
  scfg.pair_cost = ctx->opts.support_pair_cost;
  scfg.range_work = ctx->opts.support_range_work;
  scfg.stage_max = ctx->opts.support_stage_max;
  tr::SupportOut so;
  TR_TRY(tr::run_support(A, g, scfg, &so, s));
  st.triangles = so.entries / 3;
  int32_t *psi = A.get<int32_t>(g.m), *top = A.get<int32_t>(g.m);
  int32_t *cs = A.get<int32_t>(g.m), *cd = A.get<int32_t>(g.m), *ce = A.get<int32_t>(g.m);
  int32_t *phi_rows = A.get<int32_t>(g.m);
  if (!psi || !top || !cs || !cd || !ce || !phi_rows) return TRUSS_ENOMEM;
  TR_TRY(tr::compute_psi(A, g, so.sup, psi, s));
  std::vector<int64_t> cnt_ge;
  TR_TRY(tr::psi_counts(A, g.m, psi, &cnt_ge, s));
  sg.mark();  // 1: build, support, psi
  const int32_t psi_max = (int32_t)cnt_ge.size() - 1;
  int32_t kmax = 0, thr = 2;
  int64_t mc = 0;
  int rounds = 0;
  tr::PeelResult pr;
  if (g.m > 0) {
    // A non-empty k-truss has every vertex of degree >= k-1 in it, hence at
    // least k(k-1)/2 edges, all with psi >= k: k_max <= kb.
    int32_t kb = 2;
    for (int32_t k = psi_max; k > 2; k--)
      if ((double)cnt_ge[k] >= 0.5 * (double)k * (double)(k - 1)) {
        kb = k;
        break;
      }
    int32_t k_lo = kb - t + 1 > 2 ? kb - t + 1 : 2;
    const bool top_trace = getenv("TRUSS_TOP_TRACE") != nullptr;
    const std::vector<size_t> mk = A.mark();
    for (;;) {
      rounds++;
      A.rewind(mk);
      TR_TRY(tr::select_candidates(A, g, psi, k_lo, cs, cd, ce, &mc, s));
      int32_t kc = 0;
      if (mc > 0) {
        tr::RowsIn cin;
        cin.rows = mc;
        cin.n = g.n;
        cin.src = cs;
        cin.dst = cd;
        TR_TRY(decompose_device_rows(ctx, A, cin, nullptr, phi_rows, nullptr, 0, &pr, s));
        kc = pr.kmax;
      }
      if (top_trace) {
        TR_CUDA(cudaStreamSynchronize(s));
        fprintf(stderr, "truss_top round %d: k_lo %d candidates %lld k_max' %d\n", rounds, k_lo,
                (long long)mc, kc);
      }
      if (k_lo <= 2) {  // the candidate is the whole graph: everything is exact
        kmax = kc;
        thr = kmax - t + 1 > 2 ? kmax - t + 1 : 2;
        break;
      }
      if (kc >= k_lo) {
        kmax = kc;
        const int32_t need = kmax - t + 1 > 2 ? kmax - t + 1 : 2;
        if (need >= k_lo) {
          thr = need;
          break;
        }
        k_lo = need;
        continue;
      }
      // T_{k_lo} is empty: k_max(G) is in [kc, k_lo - 1], so kc - t + 1 is
      // low enough and the next round is the last
      const int32_t nk = kc - t + 1 < k_lo ? kc - t + 1 : k_lo - 1;
      k_lo = nk > 2 ? nk : 2;
    }
    TR_TRY(tr::top_classes(g.m, mc, ce, phi_rows, thr, top, s));
  }
  sg.mark();  // 2: candidate rounds
  OutBuf ot;
  TR_TRY(stage_out(A, truss_out, rows, &ot));
  TR_TRY(tr::scatter_rows(g, so.sup, top, nullptr, ot.dev, s));
  TR_TRY(copy_back(ot, rows, s));
  if (kmax_out) {
    if (is_device_ptr(kmax_out)) {
      TR_CUDA(cudaMemcpyAsync(kmax_out, &kmax, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    } else {
      *kmax_out = kmax;
    }
  }
  sg.mark();  // 3
  TR_CUDA(cudaStreamSynchronize(s));
  if (ctx->opts.profile && ctx->have_events) {
    st.ms_support = sg.ms(0, 1);
    st.ms_peel = sg.ms(1, 2);
    st.ms_scatter = sg.ms(2, 3);
    st.ms_total = sg.ms(0, 3);
  }
  st.kmax = kmax;
  st.levels = pr.levels;
  st.subrounds = pr.subrounds;
  st.candidates = mc;
  st.rounds = rounds;
  st.launches = tr::take_launches();
  ctx->last = st;
  return TRUSS_OK;
}

// Bottom-up decomposition under a working-set budget (Section 5).  The
// canonical edge list of the whole graph stays in device memory (a few
// bytes per edge); the decomposition pipeline, whose working set grows with
// the triangles, only ever runs on neighbourhood subgraphs of about `budget`
// edges.
//  Algorithm 3: while edges remain in G, split the vertices (in rank order)
//   into ranges whose degrees in G sum to at most the budget (one range if G
//   itself fits); decompose each range's neighbourhood subgraph H; every
//   edge of H keeps max(lower bound, truss number in H) (Lemma 1); each
//   internal edge leaves G, to Phi_2 if its bound is still 2 and to G_new
//   otherwise (bottomup.cu explains the reading of step 8).
//  Algorithm 4 with Procedure 5: for k = 3, 4, ... (skipping k below every
//   remaining lower bound), U_k = endpoints of G_new edges with lower bound
//   <= k, H = NS(U_k) in G_new; H is peeled at threshold k with its external
//   edges pinned, and the internal edges it removes are Phi_k.
// The supports come from one support pass over the whole graph.
// Neighbourhood subgraphs larger than the budget (a vertex whose
// degree alone exceeds it, or an NS(U_k) that does) are decomposed whole.
int run_bottom_up(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src,
                  const int32_t *dst, int64_t budget, int32_t *support_out, int32_t *truss_out,
                  int32_t *kmax_out, cudaStream_t s) {
  TR_CUDA(cudaSetDevice(ctx->device));
  tr::Arena &A = ctx->arena;
  A.reset();
  tr::take_launches();
  truss_run_stats st{};
  st.n = n;
  st.rows = rows;
  st.graphs = 1;
  Stage sg{ctx, s};
  sg.mark();  // 0
  tr::RowsIn in;
  in.rows = rows;
  in.n = n;
  TR_TRY(stage_in(A, src, rows, &in.src, s));
  TR_TRY(stage_in(A, dst, rows, &in.dst, s));
  TR_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), s));
  tr::Csr g;
  TR_TRY(tr::build_csr(A, in, &g, ctx->d_err, s));
  const int64_t m = g.m;
  st.m = m;
  // supports of the whole graph: the support pass needs no triangle lists,
  // so its working set is a few words per edge
  tr::SupportCfg scfg;
  scfg.sms = ctx->sms;
  scfg.pair_cost = ctx->opts.support_pair_cost;
  scfg.range_work = ctx->opts.support_range_work;
  scfg.stage_max = ctx->opts.support_stage_max;
  tr::SupportOut so;
  TR_TRY(tr::run_support(A, g, scfg, &so, s));
  st.triangles = so.entries / 3;
  const int32_t *supx = so.sup;
  int32_t *lower = A.get<int32_t>(m), *phi = A.get<int32_t>(m);
  uint8_t *state = A.get<uint8_t>(m), *inU = A.get<uint8_t>(n), *hpin = A.get<uint8_t>(m);
  int32_t *list = A.get<int32_t>(m), *deg = A.get<int32_t>(n);
  int32_t *hs = A.get<int32_t>(m), *hd = A.get<int32_t>(m), *hid = A.get<int32_t>(m);
  int32_t *truss_h = A.get<int32_t>(m);
  if (!lower || !phi || !state || !inU || !hpin || !list || !deg || !hs || !hd || !hid ||
      !truss_h)
    return TRUSS_ENOMEM;
  TR_CUDA(cudaMemsetAsync(lower, 0, sizeof(int32_t) * (m > 0 ? m : 1), s));
  TR_CUDA(cudaMemsetAsync(phi, 0, sizeof(int32_t) * (m > 0 ? m : 1), s));
  TR_CUDA(cudaMemsetAsync(state, 0, (size_t)(m > 0 ? m : 1), s));
  const std::vector<size_t> mk = A.mark();
  tr::PeelResult pr;
  int64_t subgraphs = 0, biggest = 0;
  std::vector<int32_t> hdeg((size_t)(n > 0 ? n : 1));
  // ---------------------------------------------------- Algorithm 3 ---
  // A pass whose ranges all cut every remaining edge leaves G unchanged; the
  // next pass then doubles the budget of its ranges, so that one range
  // finally holds all of G.
  int64_t part_budget = budget, last_nl = -1;
  for (;;) {
    int64_t nl = 0;
    A.rewind(mk);
    TR_TRY(tr::bu_list_state(A, m, state, 0, list, &nl, s));
    if (nl == 0) break;
    if (nl == last_nl) part_budget *= 2;
    last_nl = nl;
    TR_TRY(tr::bu_degrees(n, nl, list, g.esrc, g.adjp, deg, s));
    TR_CUDA(cudaMemcpyAsync(hdeg.data(), deg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    TR_CUDA(cudaStreamSynchronize(s));
    std::vector<std::pair<int32_t, int32_t>> parts;
    if (nl <= part_budget) {
      parts.push_back({0, (int32_t)n});
    } else {
      int64_t acc = 0;
      int32_t a = 0;
      for (int64_t v = 0; v < n; v++) {
        if (acc > 0 && acc + hdeg[v] > part_budget) {
          parts.push_back({a, (int32_t)v});
          a = (int32_t)v;
          acc = 0;
        }
        acc += hdeg[v];
      }
      parts.push_back({a, (int32_t)n});
    }
    for (auto &pt : parts) {
      const std::vector<size_t> mk2 = A.mark();
      int64_t mh = 0;
      TR_TRY(tr::bu_select_range(A, nl, list, g.esrc, g.adjp, pt.first, pt.second, hs, hd, hid,
                                 &mh, s));
      if (mh == 0) continue;
      tr::RowsIn hin;
      hin.rows = mh;
      hin.n = n;
      hin.src = hs;
      hin.dst = hd;
      TR_TRY(decompose_device_rows(ctx, A, hin, nullptr, truss_h, nullptr, 0, &pr, s));
      TR_TRY(tr::bu_alg3_update(mh, hid, hs, hd, pt.first, pt.second, truss_h, lower, phi,
                                state, s));
      subgraphs++;
      if (mh > biggest) biggest = mh;
      A.rewind(mk2);
    }
  }
  // ------------------------------------------- Algorithm 4, Procedure 5 ---
  // every truss number is at most the largest support + 2: a k beyond that
  // with edges left in G_new would mean an inconsistency
  int32_t maxsup = 0;
  TR_TRY(tr::bu_max(A, m, supx, &maxsup, s));
  int32_t kmax = 0;
  for (int32_t k = 3;; k++) {
    int64_t nl = 0;
    A.rewind(mk);
    TR_TRY(tr::bu_list_state(A, m, state, 1, list, &nl, s));
    if (nl == 0) break;
    if (k > maxsup + 2) return TRUSS_ECHECK;
    int32_t mn = 0;
    TR_TRY(tr::bu_min_lower(A, nl, list, lower, &mn, s));
    if (mn > k) k = mn;  // U_k is empty below the smallest lower bound
    if (k > maxsup + 2) return TRUSS_ECHECK;
    int64_t mh = 0;
    TR_TRY(tr::bu_select_candidates(A, n, nl, list, g.esrc, g.adjp, lower, k, inU, hs, hd, hid,
                                    hpin, &mh, s));
    tr::RowsIn hin;
    hin.rows = mh;
    hin.n = n;
    hin.src = hs;
    hin.dst = hd;
    TR_TRY(decompose_device_rows(ctx, A, hin, nullptr, truss_h, hpin, k, &pr, s));
    TR_TRY(tr::bu_assign(mh, hid, hpin, truss_h, k, phi, state, s));
    subgraphs++;
    if (mh > biggest) biggest = mh;
    kmax = k;
  }
  if (kmax == 0 && m > 0) kmax = 2;
  sg.mark();  // 1
  OutBuf os, ot;
  TR_TRY(stage_out(A, support_out, rows, &os));
  TR_TRY(stage_out(A, truss_out, rows, &ot));
  TR_TRY(tr::scatter_rows(g, supx, phi, os.dev, ot.dev, s));
  TR_TRY(copy_back(os, rows, s));
  TR_TRY(copy_back(ot, rows, s));
  if (kmax_out) {
    if (is_device_ptr(kmax_out)) {
      TR_CUDA(cudaMemcpyAsync(kmax_out, &kmax, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    } else {
      *kmax_out = kmax;
    }
  }
  sg.mark();  // 2
  TR_CUDA(cudaStreamSynchronize(s));
  if (ctx->opts.profile && ctx->have_events) {
    st.ms_peel = sg.ms(0, 1);
    st.ms_scatter = sg.ms(1, 2);
    st.ms_total = sg.ms(0, 2);
  }
  st.kmax = kmax;
  st.candidates = biggest;
  st.rounds = (int32_t)subgraphs;
  st.launches = tr::take_launches();
  ctx->last = st;
  return TRUSS_OK;
}

// Core numbers of the vertices of the graph the rows define.
int run_core_numbers(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src,
                     const int32_t *dst, int32_t *core_out, int32_t *kmax_out, cudaStream_t s) {
  TR_CUDA(cudaSetDevice(ctx->device));
  tr::Arena &A = ctx->arena;
  A.reset();
  tr::take_launches();
  truss_run_stats st{};
  st.n = n;
  st.rows = rows;
  st.graphs = 1;
  Stage sg{ctx, s};
  sg.mark();  // 0
  tr::RowsIn in;
  in.rows = rows;
  in.n = n;
  TR_TRY(stage_in(A, src, rows, &in.src, s));
  TR_TRY(stage_in(A, dst, rows, &in.dst, s));
  TR_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), s));
  tr::Csr g;
  TR_TRY(tr::build_csr(A, in, &g, ctx->d_err, s));
  st.m = g.m;
  sg.mark();  // 1
  OutBuf oc;
  TR_TRY(stage_out(A, core_out, n, &oc));
  int32_t kmax = 0, levels = 0, subrounds = 0;
  const long long wait = ctx->opts.wait_limit_ns > 0 ? ctx->opts.wait_limit_ns : 4000000000LL;
  TR_TRY(tr::run_core(A, g, ctx->sms, wait, oc.dev, &kmax, &levels, &subrounds, s));
  sg.mark();  // 2
  TR_TRY(copy_back(oc, n, s));
  if (kmax_out) {
    if (is_device_ptr(kmax_out)) {
      TR_CUDA(cudaMemcpyAsync(kmax_out, &kmax, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    } else {
      *kmax_out = kmax;
    }
  }
  TR_CUDA(cudaStreamSynchronize(s));
  if (ctx->opts.profile && ctx->have_events) {
    st.ms_build = sg.ms(0, 1);
    st.ms_peel = sg.ms(1, 2);
    st.ms_total = sg.ms(0, 2);
  }
  st.kmax = kmax;
  st.levels = levels;
  st.subrounds = subrounds;
  st.launches = tr::take_launches();
  ctx->last = st;
  return TRUSS_OK;
}

}  // namespace

namespace tr {
// Batched decomposition with per-graph distinct-edge and triangle counts
// (host arrays of G entries); used by the request server.
int decompose_batch_counts(truss_ctx *ctx, int32_t G, const int64_t *n, const int64_t *row_off,
                           const int32_t *src, const int32_t *dst, int32_t *support_out,
                           int32_t *truss_out, int32_t *kmax_out, cudaStream_t s,
                           int64_t *graph_m, int64_t *graph_tri) {
  std::vector<int64_t> voff((size_t)G + 1, 0);
  for (int32_t g = 0; g < G; g++) voff[g + 1] = voff[g] + n[g];
  const int64_t rows = row_off[G];
  if (rows == 0) {
    for (int32_t g = 0; g < G; g++) {
      if (kmax_out) kmax_out[g] = 0;
      graph_m[g] = graph_tri[g] = 0;
    }
    return TRUSS_OK;
  }
  return run_pipeline(ctx, voff[G], rows, src, dst, G, row_off, voff.data(), support_out,
                      truss_out, kmax_out, true, s, graph_m, graph_tri);
}
int ctx_device(truss_ctx *ctx) { return ctx->device; }
// Release the context's workspace if it holds more than max_bytes.
void ctx_trim(truss_ctx *ctx, size_t max_bytes) {
  if (ctx->arena.reserved() > max_bytes) {
    cudaSetDevice(ctx->device);
    ctx->arena.release_all();
  }
}
const truss_opts *ctx_opts(truss_ctx *ctx) { return &ctx->opts; }
void ctx_set_limit(truss_ctx *ctx, size_t bytes) { ctx->arena.set_limit(bytes); }
}  // namespace tr

extern "C" {

const char *truss_strerror(int code) {
  switch (code) {
    case TRUSS_OK: return "ok";
    case TRUSS_EINVAL: return "invalid argument (bad size, null pointer or vertex id out of range)";
    case TRUSS_ENOMEM: return "out of memory";
    case TRUSS_ECUDA: return "CUDA runtime error";
    case TRUSS_ETIMEOUT: return "a bounded device-side wait timed out";
    case TRUSS_EAGAIN: return "result not ready";
    case TRUSS_EBUSY: return "admission refused (queue full or over memory budget)";
    case TRUSS_ESHUTDOWN: return "server stopped";
    case TRUSS_ECHECK: return "internal consistency check failed";
    default: return "unknown error";
  }
}

int truss_ctx_create(truss_ctx **out, int device, const truss_opts *opts) {
  if (!out) return TRUSS_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return TRUSS_ECUDA;
  }
  if (device < 0 || device >= ndev) return TRUSS_EINVAL;
  truss_ctx *c = new (std::nothrow) truss_ctx();
  if (!c) return TRUSS_ENOMEM;
  c->device = device;
  if (opts) c->opts = *opts;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&c->d_err, sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return TRUSS_ECUDA;
  }
  bool ok = true;
  for (auto &e : c->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  c->have_events = ok;
  *out = c;
  return TRUSS_OK;
}

int truss_ctx_set_opts(truss_ctx *ctx, const truss_opts *opts) {
  if (!ctx || !opts) return TRUSS_EINVAL;
  ctx->opts = *opts;
  return TRUSS_OK;
}

int truss_ctx_destroy(truss_ctx *ctx) {
  if (!ctx) return TRUSS_OK;
  cudaSetDevice(ctx->device);
  if (ctx->have_events)
    for (auto &e : ctx->ev) cudaEventDestroy(e);
  cudaFree(ctx->d_err);
  ctx->arena.release_all();
  delete ctx;
  return TRUSS_OK;
}

int truss_support(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
                  int32_t *support_out, void *cuda_stream) {
  TR_TRY(check_common(ctx, n, rows, src, dst));
  if (rows > 0 && !support_out) return TRUSS_EINVAL;
  return run_pipeline(ctx, n, rows, src, dst, 1, nullptr, nullptr, support_out, nullptr, nullptr,
                      false, (cudaStream_t)cuda_stream);
}

int truss_decompose(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src,
                    const int32_t *dst, int32_t *support_out, int32_t *truss_out,
                    int32_t *kmax_out, void *cuda_stream) {
  TR_TRY(check_common(ctx, n, rows, src, dst));
  if (rows > 0 && !truss_out) return TRUSS_EINVAL;
  return run_pipeline(ctx, n, rows, src, dst, 1, nullptr, nullptr, support_out, truss_out,
                      kmax_out, true, (cudaStream_t)cuda_stream);
}

int truss_upper_bound(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src,
                      const int32_t *dst, int32_t *support_out, int32_t *psi_out,
                      void *cuda_stream) {
  TR_TRY(check_common(ctx, n, rows, src, dst));
  if (rows > 0 && !psi_out) return TRUSS_EINVAL;
  return run_upper_bound(ctx, n, rows, src, dst, support_out, psi_out,
                         (cudaStream_t)cuda_stream);
}

int truss_top(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
              int32_t t, int32_t *truss_out, int32_t *kmax_out, void *cuda_stream) {
  TR_TRY(check_common(ctx, n, rows, src, dst));
  if (t < 1 || (rows > 0 && !truss_out)) return TRUSS_EINVAL;
  return run_top(ctx, n, rows, src, dst, t, truss_out, kmax_out, (cudaStream_t)cuda_stream);
}

int truss_decompose_budget(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src,
                           const int32_t *dst, int64_t budget_edges, int32_t *support_out,
                           int32_t *truss_out, int32_t *kmax_out, void *cuda_stream) {
  TR_TRY(check_common(ctx, n, rows, src, dst));
  if (budget_edges < 1 || (rows > 0 && !truss_out)) return TRUSS_EINVAL;
  return run_bottom_up(ctx, n, rows, src, dst, budget_edges, support_out, truss_out, kmax_out,
                       (cudaStream_t)cuda_stream);
}

int truss_core(truss_ctx *ctx, int64_t n, int64_t rows, const int32_t *src, const int32_t *dst,
               int32_t *core_out, int32_t *kmax_out, void *cuda_stream) {
  TR_TRY(check_common(ctx, n, rows, src, dst));
  if (n > 0 && !core_out) return TRUSS_EINVAL;
  return run_core_numbers(ctx, n, rows, src, dst, core_out, kmax_out,
                          (cudaStream_t)cuda_stream);
}

int truss_decompose_batch(truss_ctx *ctx, int32_t G, const int64_t *n, const int64_t *row_off,
                          const int32_t *src, const int32_t *dst, int32_t *support_out,
                          int32_t *truss_out, int32_t *kmax_out, void *cuda_stream) {
  if (!ctx || G < 0 || (G > 0 && (!n || !row_off))) return TRUSS_EINVAL;
  if (G == 0) return TRUSS_OK;
  if (row_off[0] != 0) return TRUSS_EINVAL;
  std::vector<int64_t> voff((size_t)G + 1, 0);
  for (int32_t g = 0; g < G; g++) {
    if (n[g] < 0 || row_off[g + 1] < row_off[g]) return TRUSS_EINVAL;
    if (row_off[g + 1] > row_off[g] && n[g] == 0) return TRUSS_EINVAL;
    voff[g + 1] = voff[g] + n[g];
  }
  const int64_t rows = row_off[G], ntot = voff[G];
  TR_TRY(check_common(ctx, ntot > 0 ? ntot : 1, rows, src, dst));
  if (rows > 0 && !truss_out) return TRUSS_EINVAL;
  if (rows == 0) {
    if (kmax_out) {
      std::vector<int32_t> z((size_t)G, 0);
      if (is_device_ptr(kmax_out)) {
        TR_CUDA(cudaMemcpy(kmax_out, z.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice));
      } else {
        memcpy(kmax_out, z.data(), sizeof(int32_t) * G);
      }
    }
    return TRUSS_OK;
  }
  return run_pipeline(ctx, ntot, rows, src, dst, G, row_off, voff.data(), support_out, truss_out,
                      kmax_out, true, (cudaStream_t)cuda_stream);
}

int truss_last_stats(truss_ctx *ctx, truss_run_stats *out) {
  if (!ctx || !out) return TRUSS_EINVAL;
  *out = ctx->last;
  return TRUSS_OK;
}

}  // extern "C"
