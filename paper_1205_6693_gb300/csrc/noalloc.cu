// truss_support_noalloc: per-row edge support for small graphs without any
// memory allocation.
//
// Some callers cannot allocate device memory at the time they need a result:
// code running inside a memory pool or allocator callback, a host that has
// handed the whole device to another allocator, or a section that must not
// enter the CUDA allocator (and so must not synchronise with it).  For them,
// this entry point keeps all of its working memory in one fixed array that
// lives in the library's device image (file-scope `static __device__`),
// reserved on every GPU that loads the library until the process exits.
// The caller passes device-accessible input and output buffers; nothing else
// is allocated, neither here nor in a library routine.
//
// The work is the support computation of truss_support (Definition 1) done by
// one thread block: distinct edges through an open-addressing hash table,
// degrees, adjacency lists, then for each edge the common neighbours of its
// endpoints (walking the shorter list and probing the table), and finally a
// per-row lookup.  Every phase that depends on the previous one is separated
// by a block barrier, so no grid-wide synchronisation is needed.
#include <mutex>

#include "engine.h"

namespace {

constexpr int kMaxRows = TRUSS_NOALLOC_MAX_ROWS;
constexpr int kMaxN = TRUSS_NOALLOC_MAX_N;
constexpr int kSlots = 4 * kMaxRows;  // hash slots (load <= 1/4)
constexpr int kThreads = 1024;
constexpr unsigned long long kEmpty = ~0ull;

// Layout of the scratch array (element counts).
constexpr size_t kKeysBytes = sizeof(unsigned long long) * kSlots;
constexpr size_t kIntsCount = (size_t)kSlots      // edge id per slot
                              + 3 * (size_t)(kMaxN + 1)  // degree, offset, cursor
                              + 2 * (size_t)kMaxRows     // edge endpoints
                              + 2 * (size_t)kMaxRows     // adjacency
                              + (size_t)kMaxRows         // support per edge
                              + 2;                       // edge count, error flag
constexpr size_t kScratchBytes = kKeysBytes + sizeof(int32_t) * kIntsCount;

// The only working memory of truss_support_noalloc.  Shared by every call on
// a device: each call re-initialises what it reads before using it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__device__ __forceinline__ unsigned slot_of(unsigned long long key) {
  return (unsigned)((key * 0x9E3779B97F4A7C15ull) >> 40) & (kSlots - 1);
}

__device__ __forceinline__ int find_slot(const unsigned long long *keys, unsigned long long key) {
  unsigned h = slot_of(key);
  for (int probe = 0; probe < kSlots; probe++) {
    const unsigned long long k = keys[h];
    if (k == key) return (int)h;
    if (k == kEmpty) return -1;
    h = (h + 1) & (kSlots - 1);
  }
  return -1;
}

__global__ void __launch_bounds__(kThreads) k_support_noalloc(int n, int rows, const int32_t *src,
                                                              const int32_t *dst,
                                                              int32_t *support_out,
                                                              unsigned char *scratch) {
  unsigned long long *keys = (unsigned long long *)scratch;
  int32_t *ids = (int32_t *)(scratch + kKeysBytes);
  int32_t *deg = ids + kSlots;
  int32_t *off = deg + (kMaxN + 1);
  int32_t *cur = off + (kMaxN + 1);
  int32_t *eu = cur + (kMaxN + 1);
  int32_t *ev = eu + kMaxRows;
  int32_t *adj = ev + kMaxRows;
  int32_t *sup = adj + 2 * kMaxRows;
  int32_t *ctr = sup + kMaxRows;  // [0] distinct edges, [1] invalid-id flag
  const int tid = threadIdx.x;
  __shared__ int part[kThreads];

  // 0. clear everything this call reads (the array keeps the last call's data)
  for (int i = tid; i < kSlots; i += kThreads) keys[i] = kEmpty;
  for (int i = tid; i <= n; i += kThreads) {
    deg[i] = 0;
    cur[i] = 0;
  }
  if (tid == 0) {
    ctr[0] = 0;
    ctr[1] = 0;
  }
  __syncthreads();

  // 1. distinct undirected edges into the hash table
  for (int r = tid; r < rows; r += kThreads) {
    const int u = src[r], v = dst[r];
    if (u < 0 || u >= n || v < 0 || v >= n) {
      atomicExch(&ctr[1], 1);
      continue;
    }
    if (u == v) continue;
    const unsigned long long key =
        ((unsigned long long)(unsigned)min(u, v) << 32) | (unsigned)max(u, v);
    unsigned h = slot_of(key);
    for (;;) {
      const unsigned long long prev = atomicCAS(&keys[h], kEmpty, key);
      if (prev == kEmpty || prev == key) break;
      h = (h + 1) & (kSlots - 1);
    }
  }
  __syncthreads();
  if (ctr[1] != 0) return;  // vertex id out of range: the host reports it

  // 2. edge ids, endpoints and degrees
  for (int i = tid; i < kSlots; i += kThreads) {
    const unsigned long long key = keys[i];
    if (key == kEmpty) continue;
    const int id = atomicAdd(&ctr[0], 1);
    ids[i] = id;
    const int a = (int)(key >> 32), b = (int)(key & 0xFFFFFFFFu);
    eu[id] = a;
    ev[id] = b;
    atomicAdd(&deg[a], 1);
    atomicAdd(&deg[b], 1);
  }
  __syncthreads();

  // 3. adjacency offsets: exclusive prefix sum of the degrees
  const int per = (n + kThreads - 1) / kThreads;
  const int lo = min(n, tid * per), hi = min(n, lo + per);
  int s = 0;
  for (int v = lo; v < hi; v++) s += deg[v];
  part[tid] = s;
  __syncthreads();
  for (int d = 1; d < kThreads; d <<= 1) {
    const int x = tid >= d ? part[tid - d] : 0;
    __syncthreads();
    part[tid] += x;
    __syncthreads();
  }
  int acc = part[tid] - s;
  for (int v = lo; v < hi; v++) {
    off[v] = acc;
    acc += deg[v];
  }
  if (tid == kThreads - 1) off[n] = part[kThreads - 1];
  __syncthreads();

  // 4. adjacency lists
  const int m = ctr[0];
  for (int id = tid; id < m; id += kThreads) {
    const int a = eu[id], b = ev[id];
    adj[off[a] + atomicAdd(&cur[a], 1)] = b;
    adj[off[b] + atomicAdd(&cur[b], 1)] = a;
  }
  __syncthreads();

  // 5. support: common neighbours, walking the shorter list
  for (int id = tid; id < m; id += kThreads) {
    int x = eu[id], y = ev[id];
    if (deg[x] > deg[y]) {
      const int t = x;
      x = y;
      y = t;
    }
    int c = 0;
    for (int j = off[x]; j < off[x + 1]; j++) {
      const int w = adj[j];
      if (w == y) continue;
      const unsigned long long key =
          ((unsigned long long)(unsigned)min(y, w) << 32) | (unsigned)max(y, w);
      c += find_slot(keys, key) >= 0;
    }
    sup[id] = c;
  }
  __syncthreads();

  // 6. per-row output
  for (int r = tid; r < rows; r += kThreads) {
    const int u = src[r], v = dst[r];
    int out = -1;
    if (u != v) {
      const unsigned long long key =
          ((unsigned long long)(unsigned)min(u, v) << 32) | (unsigned)max(u, v);
      const int sl = find_slot(keys, key);
      out = sl >= 0 ? sup[ids[sl]] : -1;
    }
    support_out[r] = out;
  }
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

int scratch_for_current_device(unsigned char **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TRUSS_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return TRUSS_EINVAL;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return TRUSS_ECUDA;
    }
    g_scratch_addr[dev] = (unsigned char *)p;
  }
  *out = g_scratch_addr[dev];
  return TRUSS_OK;
}

// True if the kernel, launched on device `dev`, may dereference p as given:
// memory of that same device, managed memory, or pinned host memory mapped
// at the same address.  Memory of another GPU is refused (without peer
// access a kernel reading it would fault), and so is pageable host memory.
bool device_accessible(const void *p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice: return at.device == dev;
    case cudaMemoryTypeManaged: return true;
    case cudaMemoryTypeHost: return at.devicePointer == p;
    default: return false;
  }
}

}  // namespace

extern "C" int truss_support_noalloc(int64_t n, int64_t rows, const int32_t *src,
                                     const int32_t *dst, int32_t *support_out,
                                     void *cuda_stream) {
  if (n < 0 || rows < 0 || n > kMaxN || rows > kMaxRows) return TRUSS_EINVAL;
  if (rows == 0) return TRUSS_OK;
  if (!src || !dst || !support_out || n == 0) return TRUSS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return TRUSS_ECUDA;
  }
  if (!device_accessible(src, dev) || !device_accessible(dst, dev) ||
      !device_accessible(support_out, dev))
    return TRUSS_EINVAL;
  unsigned char *scratch = nullptr;
  TR_TRY(scratch_for_current_device(&scratch));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_support_noalloc<<<1, kThreads, 0, s>>>((int)n, (int)rows, src, dst, support_out, scratch);
  if (cudaGetLastError() != cudaSuccess) return TRUSS_ECUDA;
  // the invalid-id flag lives in the scratch array; read it back
  int32_t flag = 0;
  const size_t flag_off = kKeysBytes + sizeof(int32_t) * (kIntsCount - 1);
  if (cudaMemcpyAsync(&flag, scratch + flag_off, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return TRUSS_ECUDA;
  }
  return flag != 0 ? TRUSS_EINVAL : TRUSS_OK;
}
