// Kernels of the deterministic step; the device code is in events_device.cuh.
#include "events_device.cuh"

namespace episim {

size_t events_smem_bytes(int64_t n_events, int64_t n_levels, int64_t n_touched, int nc) {
  if (n_events == 0) return 0;
  return (size_t)n_events * 48 + (size_t)(n_levels + 1) * 4 + (size_t)n_touched * nc * 4 + 16;
}

namespace {

template <int NA>
__global__ void __launch_bounds__(512) k_events_day(EvArgs a) {
  events_block_global<NA>(a, blockIdx.x);
}

template <int NA>
__global__ void __launch_bounds__(kDfThreads, 4) k_events_day_df(EvDfArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  events_block_dataflow<NA>(a, (int)(blockIdx.x / (unsigned)a.nblk), (int)(blockIdx.x % (unsigned)a.nblk), smem);
}

template <int NA>
__global__ void __launch_bounds__(512, 1) k_events_day_smem(EvSmemArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  events_block_smem<NA>(a, blockIdx.x, smem);
}

}  // namespace

size_t events_df_smem_bytes(int64_t n_events, int64_t n_touched, int nc) {
  if (n_events == 0) return 0;
  return (size_t)n_events * 64 + (size_t)n_touched * (nc + 2) * 4 + (size_t)(2 * kDfThreads + 1) * 4 + 16;
}

cudaError_t launch_events_day_df(const EvDfArgs& a, int n_age, cudaStream_t st) {
  static bool attr_set[2] = {false, false};
  const int which = n_age == 1 ? 0 : 1;
  if (!attr_set[which]) {
    cudaError_t e = n_age == 1
        ? cudaFuncSetAttribute(k_events_day_df<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEventsSmemLimit)
        : cudaFuncSetAttribute(k_events_day_df<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEventsSmemLimit);
    if (e != cudaSuccess) return e;
    attr_set[which] = true;
  }
  const dim3 grid((unsigned)a.R * (unsigned)a.nblk);
  return n_age == 1
      ? launch_maybe_pdl(k_events_day_df<1>, grid, dim3(kDfThreads), (size_t)a.smem_bytes, st, a.overlap != 0, a)
      : launch_maybe_pdl(k_events_day_df<3>, grid, dim3(kDfThreads), (size_t)a.smem_bytes, st, a.overlap != 0, a);
}

cudaError_t launch_events_day(const EvArgs& a, int n_age, cudaStream_t st) {
  if (n_age == 1) k_events_day<1><<<a.R, 512, 0, st>>>(a);
  else k_events_day<3><<<a.R, 512, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_events_day_smem(const EvSmemArgs& a, int n_age, cudaStream_t st) {
  static bool attr_set[2] = {false, false};
  const int which = n_age == 1 ? 0 : 1;
  if (!attr_set[which]) {
    cudaError_t e = n_age == 1
        ? cudaFuncSetAttribute(k_events_day_smem<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEventsSmemLimit)
        : cudaFuncSetAttribute(k_events_day_smem<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEventsSmemLimit);
    if (e != cudaSuccess) return e;
    attr_set[which] = true;
  }
  if (n_age == 1) k_events_day_smem<1><<<a.R, 512, a.smem_bytes, st>>>(a);
  else k_events_day_smem<3><<<a.R, 512, a.smem_bytes, st>>>(a);
  return cudaGetLastError();
}

}  // namespace episim
