// Stochastic step (Eq. (numstep3)): Gillespie's direct method per node on
// [d, d+1) with phi frozen (Sec. 3.3, Eqs. (sampling) and (sampling2); the
// per-node loop of Alg. 1), one thread per (replicate, node).  The
// continuous-state update of the previous day (Eq. (numstep5) with Eq.
// (siminfpressure); the last step of Alg. 1's day) is fused into the prologue,
// as Alg. 2 places it at the start of the next stochastic task; the day's
// infected/total statistics are reduced there too.
//
// Arithmetic (identical, by specification, to the CPU oracle): per class j,
//   a_inf = (upsilon_j * phi) * S_j, a_rec = gamma_j * I_j, A_j = a_inf + a_rec,
//   a0 = A_1 or (A_1 + A_2) + A_3;  tau = E / a0;  stop when t + tau >= 1;
//   r = a0 * u2 selects inf_1, rec_1, inf_2, ... by left-to-right thresholds.
// IEEE binary64 operations are explicit intrinsics (never contracted).
#include <algorithm>

#include "ssa_device.cuh"

namespace episim {

template <int NA, bool SCORE, int MODE>
__global__ void __launch_bounds__(256, 1) k_node_day(SsaArgs a, int blocks_per_rep) {
  // 1-D grid: replicate r owns blocks [r * blocks_per_rep, (r + 1) * blocks_per_rep)
  const int r = (int)(blockIdx.x / (unsigned)blocks_per_rep);
  const int bx = (int)(blockIdx.x - (unsigned)r * (unsigned)blocks_per_rep);
  node_day_block<NA, SCORE, MODE>(a, r, bx);
}

template <int NA, bool SCORE>
__global__ void __launch_bounds__(SCORE ? 256 : 512, SCORE ? (NA == 1 ? 4 : 3) : 1) k_node_day_dealt(SsaArgs a) {
  grid_dependents_launch();
  grid_dependency_wait();                          // counts and phi of the previous step
  node_day_dealt<NA, SCORE>(a);
}

template <bool SCORE>
static cudaError_t launch_dealt(const SsaArgs& a, int n_age, cudaStream_t st) {
  // resident grid: G = SMs x (blocks of 8 warps an SM holds, fewer when the
  // units do not fill them); W warps per block, each looping over its units
  static int resident[2] = {0, 0};
  const int which = n_age == 1 ? 0 : 1;
  if (!resident[which]) {
    int nb = 0;
    cudaError_t e = n_age == 1
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_node_day_dealt<1, SCORE>, 256, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_node_day_dealt<3, SCORE>, 256, 0);
    if (e != cudaSuccess) return e;
    resident[which] = nb > 0 ? nb : 1;
  }
  const int64_t units =
      (int64_t)a.R * (a.n_big + (a.n_mid + 3) / 4 + (a.n_list - a.n_big - a.n_mid + 31) / 32);
  if (units == 0) return cudaSuccess;
  const int64_t sms = a.sm_count > 0 ? a.sm_count : 1;
  const int64_t wmax = a.max_warps > 0 ? a.max_warps : 8;
  const int64_t fit = a.max_per_sm > 0 ? std::min(resident[which], a.max_per_sm) : resident[which];
  const int64_t per_sm = std::max<int64_t>(1, std::min<int64_t>(fit, (units + sms * wmax - 1) / (sms * wmax)));
  const int64_t G = sms * per_sm;
  const int W = (int)std::min<int64_t>(wmax, (units + G - 1) / G);
  return n_age == 1
      ? launch_maybe_pdl(k_node_day_dealt<1, SCORE>, dim3((unsigned)G), dim3(32 * W), 0, st, a.overlap != 0, a)
      : launch_maybe_pdl(k_node_day_dealt<3, SCORE>, dim3((unsigned)G), dim3(32 * W), 0, st, a.overlap != 0, a);
}

template <int MODE>
static cudaError_t launch_impl(const SsaArgs& a, int n_age, bool score, cudaStream_t st) {
  if (MODE == 0 && a.order) return score ? launch_dealt<true>(a, n_age, st) : launch_dealt<false>(a, n_age, st);
  const int warp_blocks = (MODE == 0 && !score) ? a.warp_blocks : 0;
  const int n_thread = (MODE == 0 && !score && a.order) ? a.n_list - a.n_big : a.node_hi - a.node_lo;
  const int bpr = warp_blocks + (n_thread + 255) / 256;
  if (bpr <= 0) return cudaSuccess;                // an empty node range: nothing to run
  dim3 block(256), grid((unsigned)((int64_t)bpr * a.R));
  if (n_age == 1) {
    if (score) k_node_day<1, true, MODE><<<grid, block, 0, st>>>(a, bpr);
    else k_node_day<1, false, MODE><<<grid, block, 0, st>>>(a, bpr);
  } else {
    if (score) k_node_day<3, true, MODE><<<grid, block, 0, st>>>(a, bpr);
    else k_node_day<3, false, MODE><<<grid, block, 0, st>>>(a, bpr);
  }
  return cudaGetLastError();
}

cudaError_t launch_ssa_day(const SsaArgs& a, int n_age, bool score, cudaStream_t st) {
  return launch_impl<0>(a, n_age, score, st);
}

cudaError_t launch_finalize(const SsaArgs& a, int n_age, bool score, cudaStream_t st) {
  return launch_impl<1>(a, n_age, score, st);
}

__global__ void k_debug_neglog(const uint64_t* j, double* out, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = neglog_u(j[i]);
}

__global__ void k_debug_neglog_f32(const uint64_t* j, float* out, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = neglog_f32(j[i]);
}

__global__ void k_debug_div(const double* x, const double* y, double* out, double* ref, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { out[i] = div_pos(x[i], y[i]); ref[i] = __ddiv_rn(x[i], y[i]); }
}

cudaError_t launch_debug_div(const double* x, const double* y, double* out, double* ref, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_debug_div<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, y, out, ref, n);
  return cudaGetLastError();
}

cudaError_t launch_debug_neglog(const uint64_t* j, double* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_debug_neglog<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(j, out, n);
  return cudaGetLastError();
}

cudaError_t launch_debug_neglog_f32(const uint64_t* j, float* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_debug_neglog_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(j, out, n);
  return cudaGetLastError();
}

}  // namespace episim

namespace episim {

__global__ void k_broadcast_bytes(unsigned char* dst, const unsigned char* src, size_t bytes, int copies) {
  // dst[c * bytes + i] = src[i] for c in [0, copies); 16-byte granules when aligned
  size_t total = bytes * (size_t)copies;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i % bytes];
}

cudaError_t launch_broadcast(void* dst, const void* src, size_t bytes, int copies, cudaStream_t st) {
  if (bytes == 0 || copies <= 0) return cudaSuccess;
  k_broadcast_bytes<<<152 * 8, 256, 0, st>>>((unsigned char*)dst, (const unsigned char*)src, bytes, copies);
  return cudaGetLastError();
}

}  // namespace episim

namespace episim {

// Reverse sweep, one thread per (replicate, node); day-major storage makes
// every day's read coalesced.  Streams 24 bytes per node-day from HBM.
__global__ void __launch_bounds__(256) k_phi_backward(const double* __restrict__ traj, const DevParams* params,
                                                      double* score, int N, int R, int max_days, int ndays) {
  const int bpr = (N + 255) / 256;
  const int r = (int)(blockIdx.x / (unsigned)bpr);
  const int v = (int)(blockIdx.x - (unsigned)r * (unsigned)bpr) * blockDim.x + threadIdx.x;
  if (v >= N) return;
  const size_t plane = (size_t)max_days * R * N, stride = (size_t)R * N;
  const DevParams& p = params[r];
  double lam = 0.0, sb = 0.0, sa = 0.0;           // lambda_{d+1}
  const double* c = traj + (size_t)r * N + v;
  for (int d = ndays - 1; d >= 0; --d) {
    const size_t at = (size_t)d * stride;
    const double cd = __ldcs(c + at);
    const double ph = __ldcs(c + plane + at);
    const double q = __ldcs(c + 2 * plane + at);
    sb = __dsub_rn(sb, __dmul_rn(lam, ph));
    sa = __dadd_rn(sa, __dmul_rn(lam, q));
    lam = __dadd_rn(cd, __dmul_rn(__dadd_rn(1.0, -p.beta[season_of(d)]), lam));
  }
  double* sc = score + (size_t)r * kScoreTerms * N + v;
  sc[(size_t)6 * N] = __dadd_rn(sc[(size_t)6 * N], sb);
  sc[(size_t)7 * N] = __dadd_rn(sc[(size_t)7 * N], sa);
}

cudaError_t launch_phi_backward(const double* traj, const DevParams* params, double* score, int N, int R,
                                int max_days, int ndays, cudaStream_t st) {
  if (ndays <= 0) return cudaSuccess;
  dim3 grid((unsigned)((int64_t)((N + 255) / 256) * R));
  k_phi_backward<<<grid, 256, 0, st>>>(traj, params, score, N, R, max_days, ndays);
  return cudaGetLastError();
}

// Per-replicate score sums over nodes, fixed order: 256-thread block partials in
// a fixed tree, blocks added in index order by one thread.
__global__ void __launch_bounds__(256) k_score_sum(const double* score, int N, double* per_rep) {
  const int r = blockIdx.x / kScoreTerms, k = blockIdx.x % kScoreTerms;
  __shared__ double sh[256];
  const double* row = score + ((size_t)r * kScoreTerms + k) * N;
  double acc = 0.0;
  for (int v = threadIdx.x; v < N; v += 256) acc = __dadd_rn(acc, row[v]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) per_rep[(size_t)r * kScoreTerms + k] = sh[0];
}

__global__ void k_gradient_moments(const double* per_rep, const unsigned long long* prev_i,
                                   const unsigned long long* prev_n, const int32_t* days, int n_days, int R,
                                   int max_days, double* out) {
  const int di = blockIdx.x;
  if (di >= n_days || threadIdx.x != 0) return;
  const int d = days[di];
  double m[kMoments];
  for (int i = 0; i < kMoments; ++i) m[i] = 0.0;
  for (int r = 0; r < R; ++r) {
    const unsigned long long I = prev_i[(size_t)r * max_days + d], T = prev_n[(size_t)r * max_days + d];
    const double f = T ? __ddiv_rn((double)I, (double)T) : 0.0;
    m[0] = __dadd_rn(m[0], f);
    m[1] = __dadd_rn(m[1], __dmul_rn(f, f));
    for (int k = 0; k < kScoreTerms; ++k) {
      const double sk = per_rep[(size_t)r * kScoreTerms + k], fs = __dmul_rn(f, sk);
      m[2 + 4 * k] = __dadd_rn(m[2 + 4 * k], sk);
      m[3 + 4 * k] = __dadd_rn(m[3 + 4 * k], __dmul_rn(sk, sk));
      m[4 + 4 * k] = __dadd_rn(m[4 + 4 * k], fs);
      m[5 + 4 * k] = __dadd_rn(m[5 + 4 * k], __dmul_rn(fs, fs));
      m[2 + 4 * kScoreTerms + k] = __dadd_rn(m[2 + 4 * kScoreTerms + k], __dmul_rn(fs, sk));
    }
  }
  for (int i = 0; i < kMoments; ++i) out[(size_t)di * kMoments + i] = m[i];
}

cudaError_t launch_gradient_moments(const double* score, const unsigned long long* prev_i,
                                    const unsigned long long* prev_n, const int32_t* days, int n_days, int N,
                                    int R, int max_days, double* per_rep, double* out, cudaStream_t st) {
  k_score_sum<<<R * kScoreTerms, 256, 0, st>>>(score, N, per_rep);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_days <= 0) return e;
  k_gradient_moments<<<n_days, 32, 0, st>>>(per_rep, prev_i, prev_n, days, n_days, R, max_days, out);
  return cudaGetLastError();
}

}  // namespace episim
