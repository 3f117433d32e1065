// Seeded synthetic inputs generated on the GPU (input side only; no truss
// arithmetic).  gg_rmat_raw_cuda produces exactly the rows of gg_rmat_raw in
// gen.c: the same SplitMix64 counter-mode draws (Steele, Lea & Flood 2014)
// and the same 32-bit quadrant thresholds, two levels per draw.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ULL;

__host__ __device__ inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t sm_key(uint64_t seed, uint64_t stream) {
  return sm_mix(sm_mix(seed + kGolden) ^ (stream * kGolden + 0x632BE59BD9B4E019ULL));
}

__device__ inline uint64_t sm_at(uint64_t key, uint64_t ctr) { return sm_mix(key + (ctr + 1) * kGolden); }

__global__ void k_rmat_raw(int scale, int64_t ns, uint32_t t1, uint32_t t2, uint32_t t3,
                           uint64_t key, int32_t *src, int32_t *dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t u = 0, v = 0;
    uint64_t r = 0;
    for (int l = 0; l < scale; l++) {
      uint32_t x;
      if ((l & 1) == 0) {
        r = sm_at(key, (uint64_t)i * 32 + (uint64_t)(l >> 1));
        x = (uint32_t)(r >> 32);
      } else {
        x = (uint32_t)r;
      }
      uint32_t bu, bv;
      if (x < t1) { bu = 0; bv = 0; }
      else if (x < t2) { bu = 0; bv = 1; }
      else if (x < t3) { bu = 1; bv = 0; }
      else { bu = 1; bv = 1; }
      u = (u << 1) | bu;
      v = (v << 1) | bv;
    }
    src[i] = (int32_t)u;
    dst[i] = (int32_t)v;
  }
}

}  // namespace

extern "C" int gg_rmat_raw_cuda(int scale, int64_t ns, uint32_t t1, uint32_t t2, uint32_t t3,
                                uint64_t seed, uint64_t stream, int32_t *src, int32_t *dst,
                                void *cuda_stream) {
  if (ns <= 0) return 0;
  int64_t blocks = (ns + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_rmat_raw<<<(int)blocks, 256, 0, (cudaStream_t)cuda_stream>>>(scale, ns, t1, t2, t3,
                                                                  sm_key(seed, stream), src, dst);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
