// Shared device/host helpers of the truss library (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/truss.h"

#define TR_FULL 0xffffffffu

namespace tr {

// ------------------------------------------------------------------ host ---
// Evaluate a CUDA runtime call; on failure return TRUSS_ECUDA from the
// enclosing function (remembering the message for diagnostics).
void note_cuda_error(cudaError_t e, const char *what, const char *file, int line);
void count_launches(int k);

#define TR_CUDA(call)                                             \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) {                                      \
      ::tr::note_cuda_error(e_, #call, __FILE__, __LINE__);       \
      return e_ == cudaErrorMemoryAllocation ? TRUSS_ENOMEM : TRUSS_ECUDA; \
    }                                                             \
  } while (0)

// After a kernel launch: count it and check the launch error.
#define TR_LAUNCHED()                  \
  do {                                 \
    ::tr::count_launches(1);           \
    TR_CUDA(cudaGetLastError());       \
  } while (0)

#define TR_TRY(expr)          \
  do {                        \
    int rc_ = (expr);         \
    if (rc_ != TRUSS_OK) return rc_; \
  } while (0)

inline int grid_for(int64_t work, int block, int max_blocks) {
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

inline int bits_for(uint64_t maxval) {  // number of bits to represent maxval
  int b = 0;
  while (b < 64 && (maxval >> b) != 0) b++;
  return b;
}

// ---------------------------------------------------------------- device ---
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Inclusive prefix sum across the warp.
__device__ __forceinline__ int warp_incl_scan(int x) {
  const int l = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(TR_FULL, x, o);
    if (l >= o) x += y;
  }
  return x;
}

// Smallest lane o such that P[o] > t, for a non-decreasing per-lane value P
// with t < P[31].  All 32 lanes must call it.
__device__ __forceinline__ int warp_owner(int P, int t) {
  int o = 0;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    int pv = __shfl_sync(TR_FULL, P, o + s - 1);
    if (pv <= t) o += s;
  }
  return o;
}

// Warp-aggregated append: every lane with `pred` gets a distinct slot in a
// buffer whose fill counter is *cnt; returns the slot (or -1).  All lanes of
// the warp must call it.
__device__ __forceinline__ int warp_append(bool pred, int *cnt) {
  unsigned mask = __ballot_sync(TR_FULL, pred);
  if (mask == 0) return -1;
  int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane_id() == leader) base = atomicAdd(cnt, __popc(mask));
  base = __shfl_sync(TR_FULL, base, leader);
  if (!pred) return -1;
  return base + __popc(mask & ((1u << lane_id()) - 1u));
}

// As warp_append, for a monotonically increasing 64-bit counter: returns the
// counter value reserved for this lane (the caller subtracts its base).
__device__ __forceinline__ long long warp_append64(bool pred, unsigned long long *cnt) {
  unsigned mask = __ballot_sync(TR_FULL, pred);
  if (mask == 0) return -1;
  int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane_id() == leader) base = atomicAdd(cnt, (unsigned long long)__popc(mask));
  base = __shfl_sync(TR_FULL, base, leader);
  if (!pred) return -1;
  return (long long)(base + __popc(mask & ((1u << lane_id()) - 1u)));
}

// Acquire-release atomic add and acquire load at GPU scope.
__device__ __forceinline__ unsigned long long atom_add_acq_rel_gpu(unsigned long long *p,
                                                                   unsigned long long v) {
  unsigned long long old;
  asm volatile("atom.acq_rel.gpu.global.add.u64 %0, [%1], %2;"
               : "=l"(old)
               : "l"(p), "l"(v)
               : "memory");
  return old;
}

__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of a cooperative launch, with a time limit.  Arrival is
// one atomic increment of `bar`, a counter that is never reset: the block
// whose increment returned `old` waits until the counter reaches the next
// multiple of the grid size (every block arrives exactly once per barrier,
// so one barrier's arrivals are gridDim.x consecutive values).  The block's
// writes are published by the __syncthreads and the release half of the
// increment, and the other blocks' writes are seen through the acquire
// loads of the wait (or the acquire half of the last increment).  A wait
// longer than wait_ns records TRUSS_ETIMEOUT in *err.  Returns false if any
// block has recorded an error, so that every block leaves at its next
// barrier.
__device__ __forceinline__ bool grid_barrier(unsigned long long *bar, int *err,
                                             long long wait_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long old = atom_add_acq_rel_gpu(bar, 1ull);
    const unsigned long long target = (old / gridDim.x + 1) * gridDim.x;
    if (old + 1 != target) {
      volatile int *verr = err;
      const unsigned long long t0 = global_ns();
      for (unsigned spins = 1; ld_acquire_gpu(bar) < target; spins++) {
        if (spins > 32) __nanosleep(32);
        if ((spins & 15) == 0) {
          if (*verr != 0) break;
          if ((long long)(global_ns() - t0) > wait_ns) {
            atomicExch(err, TRUSS_ETIMEOUT);
            break;
          }
        }
      }
    }
    s_ok = (*(volatile int *)err) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace tr
