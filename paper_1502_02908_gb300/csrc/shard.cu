// Exchange kernels of the node-sharded single replicate (sim_shard,
// sim_pack_touched, sim_unpack_touched).
//
// Each rank holds the whole state but runs the stochastic step and the phi update
// (Eqs. (numstep3), (numstep5)) only for its own contiguous node range; every rank
// applies the whole day's event list (Eq. (numstep4)).  Between the two, the herds
// the day's events touch must hold their post-stochastic-step counts on every
// rank: each rank packs those herds' counts, the ranks gather the packs in rank
// order, and each rank takes every touched herd's counts from the pack of the rank
// that owns it.  This is the daily exchange of Sec. 3.4's crossing events, made
// over the touched herds rather than over a split of the event list.
#include "internal.h"

namespace episim {
namespace {

// out [R][Nc][n_t] = counts of the n_t touched herds (plane = r * Nc + c).
__global__ void __launch_bounds__(256) k_pack_touched(const int32_t* __restrict__ counts,
                                                       const int32_t* __restrict__ touched, int n_t, int N,
                                                       int64_t planes, int32_t* __restrict__ out) {
  const int64_t total = planes * n_t;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t plane = i / n_t;
    const int t = (int)(i - plane * n_t);
    out[i] = counts[plane * N + touched[t]];
  }
}

// counts of touched herd v = the pack of v's owner: in [world][R][Nc][n_t];
// bounds [world + 1] (rank k owns [bounds[k], bounds[k+1])); the owner is the
// largest k with bounds[k] <= v, which skips ranks with empty ranges.
__global__ void __launch_bounds__(256) k_unpack_touched(int32_t* __restrict__ counts,
                                                         const int32_t* __restrict__ touched, int n_t, int N,
                                                         int64_t planes, const int32_t* __restrict__ in,
                                                         const int32_t* __restrict__ bounds, int world) {
  const int64_t total = planes * n_t;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t plane = i / n_t;
    const int t = (int)(i - plane * n_t);
    const int v = touched[t];
    int lo = 0, hi = world - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (bounds[mid] <= v) lo = mid; else hi = mid - 1;
    }
    counts[plane * N + v] = in[(int64_t)lo * total + i];
  }
}

unsigned grid_for(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t launch_pack_touched(const int32_t* counts, const int32_t* touched, int n_t, int N, int64_t planes,
                                int32_t* out, cudaStream_t st) {
  if (n_t <= 0 || planes <= 0) return cudaSuccess;
  k_pack_touched<<<grid_for(planes * n_t), 256, 0, st>>>(counts, touched, n_t, N, planes, out);
  return cudaGetLastError();
}

cudaError_t launch_unpack_touched(int32_t* counts, const int32_t* touched, int n_t, int N, int64_t planes,
                                  const int32_t* in, const int32_t* bounds, int world, cudaStream_t st) {
  if (n_t <= 0 || planes <= 0) return cudaSuccess;
  k_unpack_touched<<<grid_for(planes * n_t), 256, 0, st>>>(counts, touched, n_t, N, planes, in, bounds, world);
  return cudaGetLastError();
}

}  // namespace episim
