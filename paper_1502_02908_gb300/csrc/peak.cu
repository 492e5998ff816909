// FP64 pipe throughput microbenchmark (sim_fp64_peak): the denominator of the
// stochastic step's arithmetic roofline.  The paper has no counterpart; its
// kernels are CPU code.  Every thread runs kChains independent dependency chains
// of one binary64 instruction kind (fused multiply-add, or add), so each
// sub-partition always has independent FP64 instructions to issue and the pipe,
// not latency, bounds the loop.  The grid is a whole number of waves: blocks per
// SM from the occupancy API times the SM count.  The chains' results are stored,
// so nothing is optimised away.
#include "../../include/episim.h"
#include "internal.h"

namespace episim {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kThreads) k_fp64_peak(const double* __restrict__ in, double* __restrict__ out,
                                                         long long iters) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double x[kChains];
  const double a = in[0], b = in[1];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = in[2 + c] + (double)t * 1e-9;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if (KIND == 0) x[c] = __fma_rn(x[c], a, b);
      else x[c] = __dadd_rn(x[c], b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s = __dadd_rn(s, x[c]);
  out[t] = s;
}

template <int KIND>
cudaError_t run(long long iters, double* lane_ops_per_s, double* ms_out) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_peak<KIND>, kThreads, 0);
  if (e != cudaSuccess) return e;
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  const size_t nthreads = (size_t)grid * kThreads;
  double* d_in = nullptr;
  double* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double h_in[2 + kChains] = {0.999999, 1e-7};
  for (int c = 0; c < kChains; ++c) h_in[2 + c] = 0.5 + 0.01 * c;
  e = cudaMalloc(&d_in, sizeof h_in);
  if (e == cudaSuccess) e = cudaMalloc(&d_out, nthreads * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(d_in, h_in, sizeof h_in, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {     // the first launch warms up
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
      k_fp64_peak<KIND><<<grid, kThreads>>>(d_in, d_out, iters);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_in);
  cudaFree(d_out);
  if (e != cudaSuccess) return e;
  const double ops = (double)nthreads * (double)iters * kChains;
  *lane_ops_per_s = ops / (best * 1e-3);
  if (ms_out) *ms_out = best;
  return cudaSuccess;
}

}  // namespace
}  // namespace episim

extern "C" sim_status sim_fp64_peak(int32_t kind, int64_t iters, double* lane_ops_per_s, double* ms) {
  if ((kind != 0 && kind != 1) || iters < 1 || !lane_ops_per_s) return SIM_E_INVALID_ARG;
  const cudaError_t e = kind == 0 ? episim::run<0>(iters, lane_ops_per_s, ms) : episim::run<1>(iters, lane_ops_per_s, ms);
  return e == cudaSuccess ? SIM_OK : SIM_E_CUDA;
}
