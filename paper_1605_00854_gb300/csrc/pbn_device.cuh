/*
 * pbn_device.cuh -- device helpers shared by the interpreter kernel (pbn_sim.cu)
 * and the per-plan kernels that the library generates and compiles at run time
 * (pbn_jit.cpp embeds this file's text as an in-memory NVRTC header).  Host code
 * includes it for pbn_jit_params only.
 */
#ifndef PBN_DEVICE_CUH
#define PBN_DEVICE_CUH

#if defined(__CUDACC_RTC__)
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned long long uint64_t;
typedef unsigned char uint8_t;
#else
#include <stdint.h>
#endif

#define PBN_JIT_MAX_ROWS 128 /* state rows a compiled plan's meta-state arrays cover */
#define PBN_DOM_PERT 1u /* Philox counter domains (c3 = domain << 28 | index) */
#define PBN_DOM_SEL 2u
#define PBN_DOM_INIT 3u
#define PBN_DOM_GEO 4u

/* Launch parameters of a compiled plan kernel. */
typedef struct {
    const uint8_t* image;        /* device copy of the plan image */
    uint64_t* state;             /* [W64][n_traj] */
    uint64_t* counts;            /* [5][n_traj] or null */
    unsigned long long* pooled;  /* [5] or null */
    uint32_t* status;            /* or null */
    uint64_t* trace;             /* [n_steps][W64][n_traj] or null */
    uint64_t traj_begin;
    uint64_t step_begin;
    uint32_t key0[10];           /* Philox key schedule: round r uses seed + r * Weyl */
    uint32_t key1[10];
    uint32_t n_traj, n_steps;
    uint32_t kv0, kp0, pairs, count_first, init;
    uint32_t trace_stride;       /* steps between trace snapshots (>= 1) */
    uint32_t tab_bytes;          /* bytes of the tables section staged into shared memory (0: read global) */
    uint32_t off_tables, off_ret, off_pos, image_bytes;
    uint32_t meta_mask[PBN_JIT_MAX_ROWS];  /* meta-state mask and value per 32-bit state row */
    uint32_t meta_val[PBN_JIT_MAX_ROWS];
} pbn_jit_params;

#if defined(__CUDACC__)

#define PBN_PHILOX_M0 0xD2511F53u
#define PBN_PHILOX_M1 0xCD9E8D57u

/* Philox4x32-10, round: (x0, x1, x2, x3) -> (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2),
 * hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)), key bumped by the Weyl constants between rounds.
 * Within one (trajectory, step) the counter words c0, c1, c2 are fixed and only
 * c3 = domain << 28 | index changes; c3 enters round 1 only through an XOR, so
 * round 1's products are computed once per step (pbn_philox_begin). */
struct pbn_philox_step {
    uint32_t y0, y1, y2b, y3;
};

template <class PT>
__device__ __forceinline__ pbn_philox_step pbn_philox_begin(const PT& P, uint64_t traj, uint64_t t) {
    const uint32_t c0 = (uint32_t)traj;
    const uint32_t c1 = (uint32_t)t;
    const uint32_t c2 = (uint32_t)((t >> 32) & 0xFFFFu) | ((uint32_t)((traj >> 32) & 0xFFFFu) << 16);
    const uint64_t p0 = (uint64_t)PBN_PHILOX_M0 * c0;
    const uint64_t p1 = (uint64_t)PBN_PHILOX_M1 * c2;
    pbn_philox_step s;
    s.y0 = (uint32_t)(p1 >> 32) ^ c1 ^ P.key0[0];
    s.y1 = (uint32_t)p1;
    s.y2b = (uint32_t)(p0 >> 32) ^ P.key1[0];
    s.y3 = (uint32_t)p0;
    return s;
}

template <class PT>
__device__ __forceinline__ uint4 pbn_philox_draw(const PT& P, const pbn_philox_step& s, uint32_t c3) {
    uint32_t x0 = s.y0, x1 = s.y1, x2 = s.y2b ^ c3, x3 = s.y3;
#pragma unroll
    for (int r = 1; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)PBN_PHILOX_M0 * x0;
        const uint64_t p1 = (uint64_t)PBN_PHILOX_M1 * x2;
        x0 = (uint32_t)(p1 >> 32) ^ x1 ^ P.key0[r];
        x2 = (uint32_t)(p0 >> 32) ^ x3 ^ P.key1[r];
        x1 = (uint32_t)p1;
        x3 = (uint32_t)p0;
    }
    return make_uint4(x0, x1, x2, x3);
}

/* ---- mbarrier + bulk copy (global -> shared) ------------------------------------ */
__device__ __forceinline__ uint32_t pbn_smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void pbn_mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(pbn_smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

/* Orders this thread's earlier generic-proxy accesses to shared memory before later
 * async-proxy operations (bulk copies) that a barrier orders after them. */
__device__ __forceinline__ void pbn_fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void pbn_mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(pbn_smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ void pbn_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            pbn_smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(pbn_smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool pbn_mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(pbn_smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

/* Bounded wait for phase 0 of a staging barrier: gives up after ~2^22 polls. */
__device__ __forceinline__ bool pbn_stage_wait(uint64_t* bar) {
    for (uint32_t it = 0; it < (1u << 22); ++it) {
        if (pbn_mbar_try_wait(bar, 0)) return true;
        if (it > 64) __nanosleep(128);
    }
    return false;
}

/* Stage `bytes` (multiple of 16, 16-byte aligned source) into dst with bulk copies
 * issued by thread 0; every thread of the CTA waits (bounded).  Returns false in
 * every thread if the copy did not complete; the copies in flight are then given a
 * second bounded wait before the caller returns. */
__device__ __forceinline__ bool pbn_stage(uint8_t* dst, const uint8_t* src, uint32_t bytes, uint64_t* bar) {
    if (threadIdx.x == 0) pbn_mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        pbn_mbar_arrive_expect_tx(bar, bytes);
        for (uint32_t off = 0; off < bytes; off += 65536u) {
            const uint32_t sz = (bytes - off) < 65536u ? (bytes - off) : 65536u;
            pbn_bulk_g2s(dst + off, src + off, sz, bar);
        }
    }
    const bool ok = pbn_stage_wait(bar);
    if (__syncthreads_or(!ok)) {
        pbn_stage_wait(bar);
        return false;
    }
    return true;
}

#endif /* __CUDACC__ */
#endif /* PBN_DEVICE_CUH */
