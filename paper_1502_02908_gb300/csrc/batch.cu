// Launch side of the persistent batch kernel: picks the instantiation of the
// requested block shape (batch_kernel.cuh, one translation unit per shape).
#include "batch.h"

namespace episim {

namespace {

BatchKernel batch_kernel(BatchShape s, bool score_any) {
  switch (s) {
    case BatchShape::k256x1: return batch_kernel_256x1(score_any);
    case BatchShape::k256x2: return batch_kernel_256x2(score_any);
    case BatchShape::k128x4: return batch_kernel_128x4(score_any);
  }
  return nullptr;
}

cudaError_t allow_smem(BatchKernel k) {
  return cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEventsSmemLimit);
}

}  // namespace

cudaError_t launch_batch(const BatchCtl& c, BatchShape s, bool score_any, int grid, cudaStream_t st) {
  const BatchKernel k = batch_kernel(s, score_any);
  cudaError_t e = allow_smem(k);
  if (e != cudaSuccess) return e;
  BatchCtl arg = c;
  void* args[] = {&arg};
  return cudaLaunchKernel((const void*)k, dim3(grid), dim3(batch_threads(s)), args, (size_t)c.smem_cap, st);
}

cudaError_t batch_occupancy(BatchShape s, bool score_any, int smem_bytes, int* blocks_per_sm) {
  const BatchKernel k = batch_kernel(s, score_any);
  cudaError_t e = allow_smem(k);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void*)k, batch_threads(s), smem_bytes);
}

}  // namespace episim
