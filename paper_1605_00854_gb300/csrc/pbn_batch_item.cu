/*
 * pbn_batch_item.cu -- the interpreter's work-item function as relocatable device
 * code.  The library builds it once (nvcc -rdc, sm_103a) next to libpbn.so; the
 * batch modules generated for batches with compiled networks are linked against it
 * at run time (nvJitLink), so that one persistent launch runs compiled networks
 * with their own code and the others with the interpreter.
 */
#include "pbn_batch_interp.cuh"

extern "C" __device__ bool pbn_batch_interp_item(uint64_t step_offset, uint32_t n_steps, const pbn_workitem* W,
                                                 const pbn_netdesc* D, const uint32_t* meta_sh, uint32_t* c,
                                                 const uint8_t* kernel_smem, uint32_t* status) {
    /* the kernel's dynamic shared memory (the staged image and trajectory rows),
     * named here so that its accesses are shared-memory accesses; the caller passes
     * its own address of it, and an item whose two addresses differ is skipped */
    extern __shared__ __align__(128) uint8_t pbn_item_smem[];
    if (static_cast<const uint8_t*>(pbn_item_smem) != kernel_smem) {
        if (status) atomicOr(status, PBN_BATCH_BAD_MODULE);
        return false;
    }
    return pbn_batch_interp_run(step_offset, n_steps, *W, *D, pbn_item_smem, meta_sh, c);
}
