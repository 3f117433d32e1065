// CUB (CCCL, header-only) device-wide radix sort and prefix sums used by the
// CSR build and the triangle-list offsets.  Kept in one translation unit so
// the heavy template instantiations compile in parallel with the kernels.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "engine.h"

namespace tr {

namespace {
// Kernels one CUB call launches: a sort is a histogram pass, a scan of the
// histograms and one onesweep pass per 8-bit digit (a single tile for small
// inputs); a scan is an init kernel plus the scan kernel.
int sort_launches(int64_t n, int bits) {
  if (n <= 4096) return 1;
  return 2 + (bits + 7) / 8;
}

int check(cudaError_t e, const char *what) {
  if (e != cudaSuccess) {
    note_cuda_error(e, what, __FILE__, __LINE__);
    return TRUSS_ECUDA;
  }
  return TRUSS_OK;
}
}  // namespace

int sort_pairs_u64(void *tmp, size_t *tmp_bytes, const uint64_t *kin, uint64_t *kout,
                   const int32_t *vin, int32_t *vout, int64_t n, int begin_bit, int end_bit,
                   cudaStream_t s) {
  if (n > INT32_MAX) return TRUSS_EINVAL;
  if (tmp) count_launches(sort_launches(n, end_bit - begin_bit));
  return check(cub::DeviceRadixSort::SortPairs(tmp, *tmp_bytes, kin, kout, vin, vout, (int)n,
                                               begin_bit, end_bit, s),
               "SortPairs<u64>");
}

int sort_keys_u64(void *tmp, size_t *tmp_bytes, const uint64_t *kin, uint64_t *kout, int64_t n,
                  int begin_bit, int end_bit, cudaStream_t s) {
  if (n > INT32_MAX) return TRUSS_EINVAL;
  if (tmp) count_launches(sort_launches(n, end_bit - begin_bit));
  return check(cub::DeviceRadixSort::SortKeys(tmp, *tmp_bytes, kin, kout, (int)n, begin_bit,
                                              end_bit, s),
               "SortKeys<u64>");
}

int sort_pairs_u32(void *tmp, size_t *tmp_bytes, const uint32_t *kin, uint32_t *kout,
                   const int32_t *vin, int32_t *vout, int64_t n, int begin_bit, int end_bit,
                   cudaStream_t s) {
  if (n > INT32_MAX) return TRUSS_EINVAL;
  if (tmp) count_launches(sort_launches(n, end_bit - begin_bit));
  return check(cub::DeviceRadixSort::SortPairs(tmp, *tmp_bytes, kin, kout, vin, vout, (int)n,
                                               begin_bit, end_bit, s),
               "SortPairs<u32>");
}

int inclusive_sum_i32(void *tmp, size_t *tmp_bytes, const int32_t *in, int32_t *out, int64_t n,
                      cudaStream_t s) {
  if (n > INT32_MAX) return TRUSS_EINVAL;
  if (tmp) count_launches(2);
  return check(cub::DeviceScan::InclusiveSum(tmp, *tmp_bytes, in, out, (int)n, s),
               "InclusiveSum<i32>");
}

int exclusive_sum_i64(void *tmp, size_t *tmp_bytes, const int64_t *in, int64_t *out, int64_t n,
                      cudaStream_t s) {
  if (n > INT32_MAX) return TRUSS_EINVAL;
  if (tmp) count_launches(2);
  return check(cub::DeviceScan::ExclusiveSum(tmp, *tmp_bytes, in, out, (int)n, s),
               "ExclusiveSum<i64>");
}

}  // namespace tr
