// The persistent batch kernels of one lag-word class W (lane, warp and CTA
// mode) and their launch helpers.  Compiled once per class with -DPSAW_W=W
// (1..8) so that the classes build in parallel.
#include "batch_device.cuh"

#ifndef PSAW_W
#error "batch_class.cu is compiled once per lag-word class with -DPSAW_W=1..8"
#endif

namespace psaw {

// dynamic shared memory of a block: one mask table per warp
template <int W>
static size_t batch_smem_bytes(int block) {
  return (size_t)(block / 32) * kBatchWarpWords<W> * sizeof(uint32_t);
}

template <int W, int U>
static cudaError_t set_batch_smem(int block) {
  return cudaFuncSetAttribute(batch_kernel<W, U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)batch_smem_bytes<W>(block));
}

template <int W>
static size_t batch_warp_smem_bytes(int block) {
  return (size_t)(block / 32) * kBatchWalkWarpWords<W> * sizeof(uint32_t);
}

template <int W>
static cudaError_t launch_batch_warp_w(int block, const BatchKernelParams &p, cudaStream_t s, int max_blocks) {
  const size_t smem = batch_warp_smem_bytes<W>(block);
  cudaError_t e = cudaFuncSetAttribute(batch_kernel_warp<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_warp<W>, block, smem)) != cudaSuccess)
    return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  int grid = per_sm * sms;
  if (max_blocks > 0 && max_blocks < grid) grid = max_blocks;
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  batch_kernel_warp<W><<<grid, block, smem, s>>>(p);
  return cudaGetLastError();
}

template <int W>
static int resident_warps_w(int block) {
  const size_t smem = batch_warp_smem_bytes<W>(block);
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaFuncSetAttribute(batch_kernel_warp<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_warp<W>, block, smem) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return per_sm * sms * (block / 32);
}

// CTA mode: blocks of kWalkBlock threads, one walk (and one visited table) each
template <int W>
static size_t batch_cta_smem_bytes() {
  return (size_t)kBatchWalkCtaWords<W> * sizeof(uint32_t);
}

template <int W>
static int resident_ctas_w() {
  const size_t smem = batch_cta_smem_bytes<W>();
  int per_sm = 0, dev = 0, sms = 0;
  if (cudaFuncSetAttribute(batch_kernel_cta<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_cta<W>, kWalkBlock, smem) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return per_sm * sms;
}

template <int W>
static cudaError_t launch_batch_cta_w(const BatchKernelParams &p, cudaStream_t s, int max_blocks) {
  int grid = resident_ctas_w<W>();
  if (max_blocks > 0 && max_blocks < grid) grid = max_blocks;
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  batch_kernel_cta<W><<<grid, kWalkBlock, batch_cta_smem_bytes<W>(), s>>>(p);
  return cudaGetLastError();
}

template <int W, int U>
static cudaError_t launch_batch_w(int block, const BatchKernelParams &p, cudaStream_t s, int *grid_out,
                                  int max_blocks) {
  int per_sm = 0;
  cudaError_t e = set_batch_smem<W, U>(block);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<W, U>, block, batch_smem_bytes<W>(block));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  int grid = per_sm * sms;
  if (max_blocks > 0 && max_blocks < grid) grid = max_blocks;
  if (grid_out) *grid_out = grid;
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  batch_kernel<W, U><<<grid, block, batch_smem_bytes<W>(block), s>>>(p);
  return cudaGetLastError();
}

template <int W, int U>
static int resident_w(int block) {
  int per_sm = 0, dev = 0, sms = 0;
  if (set_batch_smem<W, U>(block) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<W, U>, block, batch_smem_bytes<W>(block)) !=
      cudaSuccess)
    return 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return per_sm * sms * block;
}

// variant: kBatchLane (one walk per lane), kBatchLaneUnroll2 (the same with the
// scan's flip loop unrolled twice), kBatchWarp (one walk per warp) or kBatchCta
// (one walk per CTA of kWalkBlock threads; `block` is ignored)
template <int W>
cudaError_t launch_batch_class(int block, const BatchKernelParams &p, cudaStream_t s, int *grid_out, int max_blocks,
                               int variant) {
  if (variant == kBatchCta) return launch_batch_cta_w<W>(p, s, max_blocks);
  if (variant == kBatchWarp) return launch_batch_warp_w<W>(block, p, s, max_blocks);
  if (variant == kBatchLaneUnroll2) return launch_batch_w<W, 2>(block, p, s, grid_out, max_blocks);
  return launch_batch_w<W, 1>(block, p, s, grid_out, max_blocks);
}

template <int W>
int batch_resident_class(int block, int variant) {
  if (variant == kBatchCta) return resident_ctas_w<W>();
  if (variant == kBatchWarp) return resident_warps_w<W>(block);
  if (variant == kBatchLaneUnroll2) return resident_w<W, 2>(block);
  return resident_w<W, 1>(block);
}

template cudaError_t launch_batch_class<PSAW_W>(int, const BatchKernelParams &, cudaStream_t, int *, int, int);
template int batch_resident_class<PSAW_W>(int, int);

}  // namespace psaw
