// sim_gradient_moments_noalloc: the gradient-moment reduction of
// sim_gradient_moments, for callers that must not allocate device memory.
//
// Who needs it: code whose device memory is owned by someone else's allocator
// (a framework's caching pool, or an application with a fixed memory budget that
// every allocation must go through), and latency-sensitive loops where an
// allocation can synchronise the device or fragment memory.  The regular entry
// point allocates its scratch on first use; this one allocates nothing.
//
// How: the scratch it needs (per-replicate score sums, the moment sums and the
// list of days) lives in one file-scope __device__ array of fixed size, present
// on every GPU that loads the library until the process exits.  Host code cannot
// use the array's name as a device address (on the host it names a stand-in), so
// every call asks the runtime for the array's address on the current device (the
// handle's device, as for every call on a handle) with cudaGetSymbolAddress.  Nothing is cached: a cached
// pointer would go stale if the device's context were torn down and rebuilt
// (cudaDeviceReset), which reloads the library's device image elsewhere.  With
// lazy module loading (the CUDA default) the runtime places the array in device
// memory on the first lookup on a device, so the first call on each device may
// load it; make that first call before any stream capture and before measuring
// free memory.  Limits: at most kMaxReplicates replicates and kMaxDays days per
// call; larger requests are refused with SIM_E_INVALID_ARG.  All calls share the
// one array: calls that overlap on the GPU (for example on two streams) race and
// must be serialised by the caller.  Every word the kernels read from the array
// is written earlier in the same call, so nothing needs clearing between calls.
#include "../../include/episim.h"
#include "internal.h"

#include <cstdio>

namespace episim {

constexpr int kMaxReplicates = 8192;
constexpr int kMaxDays = 512;
constexpr size_t kPerRepBytes = (size_t)kMaxReplicates * kScoreTerms * sizeof(double);  // 512 KiB
constexpr size_t kMomentBytes = (size_t)kMaxDays * kMoments * sizeof(double);           // 168 KiB
constexpr size_t kDayBytes = (size_t)kMaxDays * sizeof(int32_t);                        // 2 KiB
constexpr size_t kScratchBytes = kPerRepBytes + kMomentBytes + kDayBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// Device address of the scratch array on the current device.
cudaError_t scratch_address(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

}  // namespace
}  // namespace episim

extern "C" sim_status sim_gradient_moments_noalloc(sim_handle* h, const int32_t* days, int32_t n_days,
                                                   double* per_rep, double* out, void* stream) {
  using namespace episim;
  if (!h || n_days < 0 || (n_days > 0 && (!days || !out))) return SIM_E_INVALID_ARG;
  HandleScoreView hv;
  sim_status s = handle_score_view(h, &hv);
  if (s != SIM_OK) return s;
  if (hv.R > kMaxReplicates || n_days > kMaxDays) {
    char msg[160];
    snprintf(msg, sizeof msg, "sim_gradient_moments_noalloc: %d replicates / %d days exceed its fixed scratch "
             "(at most %d replicates and %d days per call)", hv.R, n_days, kMaxReplicates, kMaxDays);
    return handle_fail(h, SIM_E_INVALID_ARG, msg);
  }
  for (int i = 0; i < n_days; ++i)
    if (days[i] < 0 || days[i] >= hv.max_days) return handle_fail(h, SIM_E_INVALID_ARG, "days out of range");
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return handle_cuda_fail(h, e, "scratch address lookup");
  double* d_per_rep = reinterpret_cast<double*>(base);
  double* d_moments = reinterpret_cast<double*>(base + kPerRepBytes);
  int32_t* d_days = reinterpret_cast<int32_t*>(base + kPerRepBytes + kMomentBytes);
  cudaStream_t st = (cudaStream_t)stream;
  if (n_days > 0) e = cudaMemcpyAsync(d_days, days, (size_t)n_days * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = launch_gradient_moments(hv.score, hv.prev_i, hv.prev_n, d_days, n_days, hv.N, hv.R, hv.max_days,
                                d_per_rep, d_moments, st);
  if (e == cudaSuccess && per_rep)
    e = cudaMemcpyAsync(per_rep, d_per_rep, (size_t)hv.R * kScoreTerms * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && n_days > 0)
    e = cudaMemcpyAsync(out, d_moments, (size_t)n_days * kMoments * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return handle_cuda_fail(h, e, "gradient moments (no-alloc)");
  return handle_check_latched(h);
}
