// Internal interfaces of the general compartment model (include/episim_general.h)
// between its host side (general_host.cpp) and its kernels (general.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace episim {

constexpr int kGenMaxComp = 16, kGenMaxTrans = 32, kGenMaxCont = 4, kGenMaxSelect = 32, kGenMaxShift = 32;
constexpr int kGenNoShift = kGenMaxShift;  // shift row of zero offsets
constexpr int kGenThreads = 128;           // threads per block of every general-model kernel
enum { kGenYPostEvent = 0, kGenYPreEvent = 1, kGenYMidpoint = 2 };

// The model as the kernels read it; every block copies it into shared memory.
struct alignas(16) GenModelDev {
  int32_t nc, nt, ny, y_source;
  int32_t fa[kGenMaxTrans], fb[kGenMaxTrans], fy[kGenMaxTrans];
  uint32_t pop[kGenMaxTrans];
  uint32_t dep[kGenMaxTrans];               // bit j of dep[n]: firing n can change rate j
  int32_t chg_off[kGenMaxTrans + 1];        // change list of transition n: chg[chg_off[n] .. chg_off[n+1])
  int32_t pad0[3];
  uint32_t chg[kGenMaxComp * kGenMaxTrans]; // (delta << 8) | compartment, delta signed
  uint32_t num[kGenMaxCont], den[kGenMaxCont];
  uint32_t select[kGenMaxSelect];
  int8_t shift[kGenMaxShift + 1][kGenMaxComp];  // row kGenNoShift is all zero
  int32_t pad1[4];
};
static_assert(sizeof(GenModelDev) % 16 == 0, "GenModelDev is copied as int4");

// Per-replicate constants.
struct alignas(16) GenRepParams {
  double rate[kGenMaxTrans];
  double alpha[kGenMaxCont];
  double beta[kGenMaxCont][4];
  double eps[kGenMaxCont];
};
static_assert(sizeof(GenRepParams) % 16 == 0, "GenRepParams is copied as int4");

struct GenSsaArgs {
  int32_t* counts;              // [R][Nc][N]
  double* y;                    // [R][Ny][N]
  double* mid;                  // midpoint variant: [R][Ny][2][N] sums U_n, D_n (else NULL)
  const GenModelDev* model;
  const GenRepParams* params;   // [R]
  const int32_t* order;         // node order (largest initial population first)
  unsigned long long* ctr;      // [R][4]
  uint64_t seed;
  int32_t rep_base, N, R, day;
  int32_t n_big;                // leading nodes of the order simulated one per warp
  int32_t n_mid;                // next nodes of the order, four per warp (8-lane segments)
  int32_t warp_blocks;          // blocks holding the warp nodes (set by the launcher)
  int32_t group_blocks;         // blocks holding the group nodes (set by the launcher)
  int32_t prologue;             // 1: first apply day - 1's continuous update (post-event or midpoint)
  uint64_t clock_margin;        // Q62 margin of the thread method's binary32 clock (0: exact method only)
};

// Event record, 16 bytes: {node, dest, count, kind | select << 8 | shift row << 16}.
struct GenEvArgs {
  int32_t* counts;
  const int4* rec;              // records grouped by (day, component), input order inside
  const int32_t* comp_ev;       // their positions in the day-stable order (Philox counter word 0)
  const int32_t* comp_off;      // [n_components + 1]
  int32_t comp0, ncomp;         // the day's components
  const GenModelDev* model;
  unsigned long long* ctr;
  int32_t* err;                 // bit 0: an event asked for absent animals (ERROR policy)
  uint64_t seed;
  int32_t rep_base, N, R, day, underflow_error;
};

struct GenContArgs {
  int32_t* counts;
  double* y;
  const double* mid;
  const GenModelDev* model;
  const GenRepParams* params;
  int32_t N, R, day;
};

size_t gen_ssa_smem_bytes(int nc, int nt);
cudaError_t launch_gen_ssa(GenSsaArgs a, int nt, int nc, cudaStream_t st);
cudaError_t launch_gen_events(const GenEvArgs& a, cudaStream_t st);
cudaError_t launch_gen_cont(const GenContArgs& a, cudaStream_t st);

}  // namespace episim
