// The persistent batch kernel with 128-thread blocks, 4 resident an SM.
#include "batch_kernel.cuh"

namespace episim {

BatchKernel batch_kernel_128x4(bool score_any) { return batch_kernel_of<128, 4>(score_any); }

}  // namespace episim
