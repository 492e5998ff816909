// The persistent batch kernel with 256-thread blocks, 2 resident an SM.
#include "batch_kernel.cuh"

namespace episim {

BatchKernel batch_kernel_256x2(bool score_any) { return batch_kernel_of<256, 2>(score_any); }

}  // namespace episim
