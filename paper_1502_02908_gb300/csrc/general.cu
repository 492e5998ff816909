// Kernels of the general compartment model (Secs. 2.1-2.2, 3.1-3.3): the
// stochastic step (direct method per node with a sparse dependency graph), the
// event step (one thread per component of the day's transfer graph) and the
// continuous update (Eqs. (numstep5) and (numstep2)).
//
// Arithmetic: rates, a0, thresholds, tau and the continuous update are binary64
// with the operation order of include/episim_general.h (no contraction; the
// build passes -fmad=false); -log(u) is the exact fixed-point logarithm of the
// SISe kernels; comparisons of non-negative doubles compare bit patterns.
#include "../../include/episim_general.h"
#include "devmath.cuh"
#include "general.h"

namespace episim {

namespace {

__device__ __forceinline__ void copy16(void* dst, const void* src, int n16) {
  int4* d = reinterpret_cast<int4*>(dst);
  const int4* s = reinterpret_cast<const int4*>(src);
  for (int i = threadIdx.x; i < n16; i += blockDim.x) d[i] = __ldg(s + i);
}

__device__ __forceinline__ double ll_to_double(long long n) { return __ll2double_rn(n); }

__device__ __forceinline__ long long mask_sum(const int32_t* x, int stride, uint32_t mask, int nc) {
  long long s = 0;
  for (int c = 0; c < nc; ++c)
    if (mask >> c & 1u) s += x[c * stride];
  return s;
}

__device__ __forceinline__ double pick(const double (&y)[kGenMaxCont], int q) {
  return q == 0 ? y[0] : q == 1 ? y[1] : q == 2 ? y[2] : y[3];
}

// a_j = k_j [* y_q] [* x_a] [* x_b] [/ P], left to right.
__device__ __forceinline__ double gen_rate(const GenModelDev& m, const GenRepParams& p, const int32_t* x,
                                           int stride, const double (&y)[kGenMaxCont], int j) {
  double a = p.rate[j];
  const int q = m.fy[j], fa = m.fa[j], fb = m.fb[j];
  const uint32_t pm = m.pop[j];
  if (q >= 0) a = __dmul_rn(a, pick(y, q));
  if (fa >= 0) a = __dmul_rn(a, i2d_exact(x[fa * stride]));
  if (fb >= 0) a = __dmul_rn(a, i2d_exact(x[fb * stride]));
  if (pm) {
    const long long P = mask_sum(x, stride, pm, m.nc);
    a = P > 0 ? __ddiv_rn(a, ll_to_double(P)) : 0.0;
  }
  return a;
}

__device__ __forceinline__ double gen_y_next(const GenModelDev& m, const GenRepParams& p, int q, int day,
                                             double y, double U, double D) {
  const double omb = __dsub_rn(1.0, p.beta[q][season_of(day)]);
  double mid;
  if (m.den[q] == 0u) mid = __dmul_rn(p.alpha[q], U);
  else mid = D > 0.0 ? __ddiv_rn(__dmul_rn(p.alpha[q], U), D) : 0.0;
  return __dadd_rn(__dadd_rn(__dmul_rn(y, omb), mid), p.eps[q]);
}

// Direct method of one node-day (Eqs. (sampling), (sampling2)); x is the node's
// counts in shared memory (stride = threads per block).
template <int NT>
__device__ __forceinline__ uint32_t gen_node_day(const GenModelDev& m, const GenRepParams& p, int32_t* x,
                                                 int stride, const double (&y)[kGenMaxCont], uint32_t v,
                                                 uint32_t day, uint32_t rep, uint32_t k0, uint32_t k1) {
  const int nt = m.nt;
  double a[NT];
#pragma unroll
  for (int j = 0; j < NT; ++j) a[j] = (j < nt) ? gen_rate(m, p, x, stride, y, j) : 0.0;
  double t = 0.0;
  uint32_t fired = 0;
  for (uint32_t k = 0;; ++k) {
    double a0 = 0.0;
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (j < nt) a0 = __dadd_rn(a0, a[j]);
    if (!pos(a0)) break;
    const uint4 w = philox10(make_uint4(v, day, k, rep), k0, k1);
    const double E = neglog_u((((uint64_t)w.y << 32) | w.x) >> 12);
    const double u2 = uniform_open(w.z, w.w);
    const double tn = __dadd_rn(t, __ddiv_rn(E, a0));
    if (le_nonneg(1.0, tn)) break;
    t = tn;
    const double r = __dmul_rn(a0, u2);
    double P = 0.0;
    int chosen = -1, last = -1;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      if (j < nt && chosen < 0) {
        P = __dadd_rn(P, a[j]);
        if (pos(a[j])) {
          last = j;
          if (le_nonneg(r, P)) chosen = j;
        }
      }
    }
    if (chosen < 0) chosen = last;
    for (int q = m.chg_off[chosen]; q < m.chg_off[chosen + 1]; ++q) {
      const uint32_t c = m.chg[q];
      x[(c & 0xffu) * stride] += (int32_t)c >> 8;
    }
    const uint32_t dm = m.dep[chosen];
#pragma unroll
    for (int j = 0; j < NT; ++j)
      if (dm >> j & 1u) a[j] = gen_rate(m, p, x, stride, y, j);
    ++fired;
  }
  return fired;
}

template <int NT>
__global__ void __launch_bounds__(kGenThreads) k_gen_ssa(GenSsaArgs a) {
  extern __shared__ int4 smem4[];
  GenModelDev& m = *reinterpret_cast<GenModelDev*>(smem4);
  GenRepParams& p = *reinterpret_cast<GenRepParams*>(reinterpret_cast<char*>(smem4) + sizeof(GenModelDev));
  int32_t* xs = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(smem4) + sizeof(GenModelDev) +
                                           sizeof(GenRepParams));
  const int r = blockIdx.y;
  copy16(&m, a.model, (int)(sizeof(GenModelDev) / 16));
  copy16(&p, a.params + r, (int)(sizeof(GenRepParams) / 16));
  __syncthreads();
  const int nc = m.nc, ny = m.ny, N = a.N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = blockDim.x;
  int32_t* x = xs + threadIdx.x;
  uint32_t fired = 0;
  if (i < N) {
    const int v = a.order[i];
    int32_t* X = a.counts + (size_t)r * nc * N;
    for (int c = 0; c < nc; ++c) x[c * stride] = X[(size_t)c * N + v];
    double y[kGenMaxCont] = {0.0, 0.0, 0.0, 0.0};
    double* Y = a.y + (size_t)r * ny * N;
#pragma unroll
    for (int q = 0; q < kGenMaxCont; ++q)
      if (q < ny) y[q] = Y[(size_t)q * N + v];
    if (m.y_source == kGenYMidpoint) {
      for (int q = 0; q < ny; ++q) {
        double* M = a.mid + ((size_t)r * ny + q) * 2 * N;
        M[v] = ll_to_double(mask_sum(x, stride, m.num[q], nc));
        M[(size_t)N + v] = ll_to_double(mask_sum(x, stride, m.den[q], nc));
      }
    }
    const uint32_t rep = (uint32_t)(a.rep_base + r);
    fired = gen_node_day<NT>(m, p, x, stride, y, (uint32_t)v, (uint32_t)a.day, rep, (uint32_t)a.seed,
                             (uint32_t)(a.seed >> 32));
    for (int c = 0; c < nc; ++c) X[(size_t)c * N + v] = x[c * stride];
    if (m.y_source == kGenYPreEvent) {
#pragma unroll
      for (int q = 0; q < kGenMaxCont; ++q)
        if (q < ny) {
          const double U = ll_to_double(mask_sum(x, stride, m.num[q], nc));
          const double D = ll_to_double(mask_sum(x, stride, m.den[q], nc));
          Y[(size_t)q * N + v] = gen_y_next(m, p, q, a.day, y[q], U, D);
        }
    }
  }
  const uint32_t tot = __reduce_add_sync(0xffffffffu, fired);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(a.ctr + (size_t)r * 4, (unsigned long long)tot);
}

// One thread per component of the day's transfer graph: its events in input
// order (no other thread touches its nodes this day).
__global__ void __launch_bounds__(kGenThreads) k_gen_events(GenEvArgs a) {
  __shared__ GenModelDev m;
  copy16(&m, a.model, (int)(sizeof(GenModelDev) / 16));
  __syncthreads();
  const int r = blockIdx.y, nc = m.nc, N = a.N;
  const int ci = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t applied = 0, clamped = 0, skipped = 0;
  if (ci < a.ncomp) {
    int32_t* X = a.counts + (size_t)r * nc * N;
    const uint32_t rep = (uint32_t)(a.rep_base + r), k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const int p1 = a.comp_off[a.comp0 + ci + 1];
    for (int pi = a.comp_off[a.comp0 + ci]; pi < p1; ++pi) {
      const int e = a.comp_ev[pi];
      const int4 rec = a.rec[e];
      const int node = rec.x, dest = rec.y, n = rec.z;
      const int kind = rec.w & 0xff, sel = (rec.w >> 8) & 0xff, sh = (rec.w >> 16) & 0xff;
      const uint32_t mask = m.select[sel];
      const int8_t* off = m.shift[sh];
      if (kind == SIM_ENTER) {
        const int c0 = __ffs(mask) - 1;
        X[(size_t)(c0 + off[c0]) * N + node] += n;
        ++applied;
        continue;
      }
      long long avail = 0;
      for (int c = 0; c < nc; ++c)
        if (mask >> c & 1u) avail += X[(size_t)c * N + node];
      int take = n;
      if ((long long)n > avail) {
        if (a.underflow_error) {
          ++skipped;
          atomicOr(a.err, 1);
          continue;
        }
        take = (int)avail;
        ++clamped;
      }
      uint4 buf = make_uint4(0, 0, 0, 0);
      uint32_t wq = 0;
      auto next = [&]() -> uint32_t {
        if ((wq & 3u) == 0u) buf = philox10(make_uint4((uint32_t)e, (uint32_t)a.day | kEventTag, wq >> 2, rep), k0, k1);
        const uint32_t s = wq & 3u;
        ++wq;
        return s == 0 ? buf.x : s == 1 ? buf.y : s == 2 ? buf.z : buf.w;
      };
      for (int t = 0; t < take; ++t) {
        uint32_t slot = lemire((uint32_t)(avail - t), next);
        int got = 0;
        for (int c = 0; c < nc; ++c) {
          if (!(mask >> c & 1u)) continue;
          const uint32_t have = (uint32_t)X[(size_t)c * N + node];
          if (slot < have) { got = c; break; }
          slot -= have;
        }
        X[(size_t)got * N + node] -= 1;
        if (kind == SIM_INTERNAL) X[(size_t)(got + off[got]) * N + node] += 1;
        else if (kind == SIM_EXTERNAL) X[(size_t)(got + off[got]) * N + dest] += 1;
      }
      ++applied;
    }
  }
  const uint32_t sa = __reduce_add_sync(0xffffffffu, applied);
  const uint32_t sc = __reduce_add_sync(0xffffffffu, clamped);
  const uint32_t ss = __reduce_add_sync(0xffffffffu, skipped);
  if ((threadIdx.x & 31) == 0) {
    unsigned long long* C = a.ctr + (size_t)r * 4;
    if (sa) atomicAdd(C + 1, (unsigned long long)sa);
    if (sc) atomicAdd(C + 2, (unsigned long long)sc);
    if (ss) atomicAdd(C + 3, (unsigned long long)ss);
  }
}

// Continuous update from the post-event counts, or the midpoint with the sums
// the stochastic step saved.
__global__ void __launch_bounds__(kGenThreads) k_gen_cont(GenContArgs a) {
  __shared__ GenModelDev m;
  __shared__ GenRepParams p;
  const int r = blockIdx.y;
  copy16(&m, a.model, (int)(sizeof(GenModelDev) / 16));
  copy16(&p, a.params + r, (int)(sizeof(GenRepParams) / 16));
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x, N = a.N, nc = m.nc, ny = m.ny;
  if (v >= N) return;
  const int32_t* X = a.counts + (size_t)r * nc * N + v;
  double* Y = a.y + (size_t)r * ny * N + v;
  for (int q = 0; q < ny; ++q) {
    double U = ll_to_double(mask_sum(X, N, m.num[q], nc));
    double D = ll_to_double(mask_sum(X, N, m.den[q], nc));
    if (m.y_source == kGenYMidpoint) {
      const double* M = a.mid + ((size_t)r * ny + q) * 2 * N + v;
      U = __dmul_rn(0.5, __dadd_rn(M[0], U));
      D = __dmul_rn(0.5, __dadd_rn(M[N], D));
    }
    Y[(size_t)q * N] = gen_y_next(m, p, q, a.day, Y[(size_t)q * N], U, D);
  }
}

}  // namespace

size_t gen_ssa_smem_bytes(int nc) {
  return sizeof(GenModelDev) + sizeof(GenRepParams) + (size_t)nc * kGenThreads * sizeof(int32_t);
}

cudaError_t launch_gen_ssa(const GenSsaArgs& a, int nt, int nc, cudaStream_t st) {
  const dim3 grid((unsigned)((a.N + kGenThreads - 1) / kGenThreads), (unsigned)a.R);
  const size_t smem = gen_ssa_smem_bytes(nc);
  if (nt <= 8) k_gen_ssa<8><<<grid, kGenThreads, smem, st>>>(a);
  else k_gen_ssa<kGenMaxTrans><<<grid, kGenThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gen_events(const GenEvArgs& a, cudaStream_t st) {
  if (a.ncomp <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((a.ncomp + kGenThreads - 1) / kGenThreads), (unsigned)a.R);
  k_gen_events<<<grid, kGenThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gen_cont(const GenContArgs& a, cudaStream_t st) {
  const dim3 grid((unsigned)((a.N + kGenThreads - 1) / kGenThreads), (unsigned)a.R);
  k_gen_cont<<<grid, kGenThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace episim
