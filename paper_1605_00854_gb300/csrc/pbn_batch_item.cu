/*
 * pbn_batch_item.cu -- the interpreter's work-item function as relocatable device
 * code.  The library builds it once (nvcc -rdc, sm_103a) next to libpbn.so; the
 * batch modules generated for batches with compiled networks are linked against it
 * at run time (nvJitLink), so that one persistent launch runs compiled networks
 * with their own code and the others with the interpreter.
 */
#include "pbn_batch_interp.cuh"

extern "C" __device__ bool pbn_batch_interp_item(uint64_t step_offset, uint32_t n_steps, const pbn_workitem* W,
                                                 const pbn_netdesc* D, const uint32_t* meta_sh, uint32_t* c) {
    /* the kernel's dynamic shared memory (the staged image and trajectory rows) */
    extern __shared__ __align__(128) uint8_t pbn_item_smem[];
    return pbn_batch_interp_run(step_offset, n_steps, *W, *D, pbn_item_smem, meta_sh, c);
}
