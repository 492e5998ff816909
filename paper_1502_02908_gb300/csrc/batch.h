// Descriptors of the persistent batch kernel (batch.cu), filled by host.cpp.
#pragma once
#include "internal.h"

namespace episim {

// Block shapes of the persistent kernel: threads a block x blocks an SM (the
// register budget).  A stochastic-step chunk is one block's worth of nodes (one a
// thread) or of large herds (one a warp), so the shape also sets the chunk size.
enum class BatchShape { k256x1, k256x2, k128x4 };
constexpr int batch_threads(BatchShape s) { return s == BatchShape::k128x4 ? 128 : 256; }
constexpr int batch_min_blocks(BatchShape s) {
  return s == BatchShape::k256x2 ? 2 : s == BatchShape::k128x4 ? 4 : 1;
}
constexpr int kBatchTimeout = 2;      // error bit: a bounded wait ran out
constexpr int kBatchSubs = 4;         // blocks' worth of per-thread nodes in a chunk

struct BatchInst {
  SsaArgs ssa;            // node order / warp split set for one block's chunks
  EvSmemArgs evs;
  EvArgs evg;
  const int32_t* day_smem;  // [max_days] shared memory of the staged event step (0: global variant)
  int32_t na, score, has_events;
  int32_t bpr;            // stochastic-step chunks per replicate
  int32_t subs;           // blocks' worth of per-thread nodes in one chunk
  int32_t n_thread;       // nodes on the per-thread path
  int32_t tbpr;           // finalisation chunks per replicate
  int32_t day0, ndays;
  unsigned* ssa_done;     // [R] chunks completed in this run
  unsigned* ev_done;      // [R] 1 + last day whose events are applied (starts at day0)
};

struct BatchCtl {
  const BatchInst* inst;  // [n_inst], longest horizon first
  const long long* cumA;  // [n_inst + 1] prefix sums of R * bpr
  const long long* cumB;  // [n_inst + 1] prefix sums of R
  const long long* cumF;  // [n_inst + 1] prefix sums of R * tbpr
  const long long* step_off;  // [n_steps + 1] first item of each step
  const int32_t* active;  // [n_steps] instances still running at each step (a prefix)
  unsigned long long* next;
  int* abort;
  int* err;
  long long total_main, total;
  long long spin_limit;
  int n_inst, n_steps;
  int smem_cap;
};

using BatchKernel = void (*)(BatchCtl);
BatchKernel batch_kernel_256x1(bool score_any);
BatchKernel batch_kernel_256x2(bool score_any);
BatchKernel batch_kernel_128x4(bool score_any);

cudaError_t launch_batch(const BatchCtl& c, BatchShape s, bool score_any, int grid, cudaStream_t st);
cudaError_t batch_occupancy(BatchShape s, bool score_any, int smem_bytes, int* blocks_per_sm);

}  // namespace episim
