// Halo exchange support for a list cut into chunks (Sec. 2: each rank
// receives the PDFs of its remote links into ghost cells before a step).
// The pack side of the exchange is a gather by slot list; on one device it
// can read a peer chunk's array and write straight into the ghost run.
#include "lbm_internal.cuh"

namespace {

template <class T>
__global__ void halo_gather_kernel(const T* __restrict__ src, const int64_t* __restrict__ slots,
                                   int64_t count, T* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = src[slots[i]];
}

}  // namespace

using namespace lbm;

extern "C" int lbm_halo_gather(const void* src_dev, const int64_t* slots_dev, int64_t count,
                               void* dst_dev, int32_t elem_bytes, void* stream) {
  clear_error();
  if (count < 0) return fail(LBM_EINVAL, "count %lld < 0", (long long)count);
  if (count == 0) return LBM_OK;
  if (!src_dev || !slots_dev || !dst_dev) return fail(LBM_EINVAL, "NULL pointer");
  const unsigned grid = (unsigned)((count + 255) / 256);
  const cudaStream_t s = (cudaStream_t)stream;
  switch (elem_bytes) {
    case 2:
      halo_gather_kernel<uint16_t><<<grid, 256, 0, s>>>((const uint16_t*)src_dev, slots_dev, count, (uint16_t*)dst_dev);
      break;
    case 4:
      halo_gather_kernel<uint32_t><<<grid, 256, 0, s>>>((const uint32_t*)src_dev, slots_dev, count, (uint32_t*)dst_dev);
      break;
    case 8:
      halo_gather_kernel<uint64_t><<<grid, 256, 0, s>>>((const uint64_t*)src_dev, slots_dev, count, (uint64_t*)dst_dev);
      break;
    default:
      return fail(LBM_EINVAL, "element size %d not in {2, 4, 8}", elem_bytes);
  }
  LBM_CUDA_TRY(cudaGetLastError());
  return LBM_OK;
}
