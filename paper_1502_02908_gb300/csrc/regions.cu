// Region statistics of the parameter-fitting goal (Sec. 4.3, Eqs. (goal),
// (goalvariance), (goalsigma)): after each day, per replicate i, region j and
// compartment c, the region total x_jc^i = sum over the region's nodes of the
// node's count; accumulated over replicates as exact integers
//   s1[d][j][c] = sum_i x_jc^i,   s2[d][j][c] = sum_i (x_jc^i)^2.
// The goal over days [d0, d0 + n) against a reference trajectory's region totals
// ref[d][j][c] (R = number of trajectories):
//   G^2  = sum_d sum_j sum_c (s1 / R - ref)^2
//   VG^2 = sum_d sum_j sum_c (s2 - s1^2 / R) / (R - 1)
// (the time integral of the paper taken over the daily observations, dt = 1).
#include "internal.h"

namespace episim {

namespace {

constexpr int kRegionThreads = 256;

// One block per (replicate, region): the region's nodes (region-sorted list) are
// summed per compartment, then the block adds the totals and their squares.
__global__ void __launch_bounds__(kRegionThreads) k_region_day(const int32_t* __restrict__ counts,
                                                               const int32_t* __restrict__ reg_nodes,
                                                               const int32_t* __restrict__ reg_off, int N, int R,
                                                               int Nc, int J, int day, unsigned long long* s1,
                                                               unsigned long long* s2) {
  __shared__ long long part[kRegionThreads / 32][6];
  const int r = (int)(blockIdx.x / (unsigned)J), j = (int)(blockIdx.x % (unsigned)J);
  long long acc[6] = {0, 0, 0, 0, 0, 0};
  const int32_t* X = counts + (size_t)r * Nc * N;
  for (int i = reg_off[j] + (int)threadIdx.x; i < reg_off[j + 1]; i += blockDim.x) {
    const int v = reg_nodes[i];
    for (int c = 0; c < Nc; ++c) acc[c] += __ldcg(X + (size_t)c * N + v);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < Nc; ++c) {
    long long v = acc[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < (unsigned)Nc) {
    const int c = threadIdx.x;
    long long tot = 0;
    for (int w = 0; w < kRegionThreads / 32; ++w) tot += part[w][c];
    const size_t at = ((size_t)day * J + j) * Nc + c;
    atomicAdd(s1 + at, (unsigned long long)tot);
    atomicAdd(s2 + at, (unsigned long long)(tot * tot));
  }
}

// One block: each thread sums its strided terms in order, then a fixed-order
// tree reduction (deterministic).  Differences and variances are formed exactly
// in 128-bit integers before the division.
__global__ void __launch_bounds__(kRegionThreads) k_goal(const unsigned long long* __restrict__ s1,
                                                         const unsigned long long* __restrict__ s2,
                                                         const long long* __restrict__ ref, long long first,
                                                         long long count, int R, double* out) {
  __shared__ double gs[kRegionThreads], vs[kRegionThreads];
  double g = 0.0, v = 0.0;
  for (long long i = threadIdx.x; i < count; i += blockDim.x) {
    const long long a = (long long)s1[first + i], b = (long long)s2[first + i];
    const __int128 diff = (__int128)a - (__int128)R * ref[i];       // R (mean - ref)
    const double d = (double)diff / (double)R;
    g = __dadd_rn(g, __dmul_rn(d, d));
    if (R > 1) {
      const __int128 m2 = (__int128)R * b - (__int128)a * a;         // R (R - 1) sigma^2, exact
      v = __dadd_rn(v, (double)m2 / ((double)R * (double)(R - 1)));
    }
  }
  gs[threadIdx.x] = g;
  vs[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRegionThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < (unsigned)s) {
      gs[threadIdx.x] = __dadd_rn(gs[threadIdx.x], gs[threadIdx.x + s]);
      vs[threadIdx.x] = __dadd_rn(vs[threadIdx.x], vs[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = gs[0]; out[1] = vs[0]; }
}

}  // namespace

cudaError_t launch_region_day(const int32_t* counts, const int32_t* reg_nodes, const int32_t* reg_off, int N, int R,
                              int Nc, int J, int day, unsigned long long* s1, unsigned long long* s2,
                              cudaStream_t st) {
  k_region_day<<<(unsigned)((int64_t)R * J), kRegionThreads, 0, st>>>(counts, reg_nodes, reg_off, N, R, Nc, J, day,
                                                                       s1, s2);
  return cudaGetLastError();
}

cudaError_t launch_goal(const unsigned long long* s1, const unsigned long long* s2, const long long* ref,
                        long long first, long long count, int R, double* out, cudaStream_t st) {
  k_goal<<<1, kRegionThreads, 0, st>>>(s1, s2, ref, first, count, R, out);
  return cudaGetLastError();
}

}  // namespace episim
