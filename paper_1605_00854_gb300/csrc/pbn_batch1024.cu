/*
 * pbn_batch1024.cu -- the library's interpreted batch kernel with CTAs of 1,024
 * threads (64 registers a thread; one CTA per SM), for batches whose networks run
 * the interpreter: twice the warps per SM of the 512-thread kernel in pbn_batch.cu,
 * for lane groups of wide networks.  Its own translation unit, so that the build
 * compiles the two instantiations in parallel.
 */
#include <cuda_runtime.h>

#include "pbn_batch_interp.cuh"

namespace {
__global__ void __launch_bounds__(1024, 1) pbn_batch_kernel_1024(const pbn_batch_params B) {
    pbn_batch_interp_kernel_body(B);
}
}  // namespace

namespace pbn {
const void* batch_kernel_1024() { return reinterpret_cast<const void*>(pbn_batch_kernel_1024); }
}  // namespace pbn
