// The persistent batch kernel with 256-thread blocks, 1 resident an SM.
#include "batch_kernel.cuh"

namespace episim {

BatchKernel batch_kernel_256x1(bool score_any) { return batch_kernel_of<256, 1>(score_any); }

}  // namespace episim
