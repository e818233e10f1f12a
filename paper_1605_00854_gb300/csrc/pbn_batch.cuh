/*
 * pbn_batch.cuh -- the batched form of Algorithm 5's ParallelSimulation: the
 * device table of a batch (per-network descriptors and work items) and the
 * persistent work-queue loop, shared by the library's batch kernel (pbn_batch.cu),
 * the interpreter's work-item function built as relocatable device code
 * (pbn_batch_item.cu) and the batch modules generated per batch for compiled
 * networks (pbn_jit.cpp embeds this file's text as an in-memory NVRTC header).
 *
 * A launch advances every network by n_steps steps from step_begin + step_offset.
 * Each CTA pops the next work item (one network's trajectory range) with one
 * atomic, bulk-copies the network's staged bytes into shared memory when they differ
 * from the ones it holds (cp.async.bulk + mbarrier, bounded wait), runs the item
 * and pools its counts (warp shuffle tree, one atomic per warp and count).  The
 * queue is two uint32 counters: the next item and the number of CTAs that found the
 * queue empty; the last CTA to leave resets both, so launches can follow each other
 * (or be replayed from a CUDA graph) without a host reset.
 */
#ifndef PBN_BATCH_CUH
#define PBN_BATCH_CUH

#include "pbn_device.cuh"

#define PBN_BATCH_META_ROWS 16
#define PBN_BATCH_STAGE_TIMEOUT 1u /* status bit: a staging copy did not complete */
#define PBN_BATCH_BAD_MODULE 4u    /* status bit: a linked function sees other shared memory */
#define PBN_WEYL0 0x9E3779B9u      /* Philox key increments between rounds */
#define PBN_WEYL1 0xBB67AE85u

/* Per-network descriptor in device memory (written by the host, read-only).  For a
 * network run by compiled code (`compiled` = 1) only the buffers, the counting
 * window, the staging fields and lg / nt are read; the code holds the rest. */
struct alignas(16) pbn_netdesc {
    const uint8_t* image;
    uint64_t* state;
    uint64_t* counts;
    unsigned long long* pooled;
    uint64_t traj_begin, step_begin, count_from, seed;
    uint32_t n_traj, init, stage_bytes, image_bytes;
    uint32_t smem_state_off, hmax, tables_in_smem, n_meta_rows;
    uint32_t n, W, W32, n_sel;
    uint32_t P, off_words, off_groups, off_multi;
    uint32_t off_selslot, off_thr, off_inputs, off_selblk;
    uint32_t off_ret, off_pos, off_tables, specs_in_smem;
    uint32_t nt, off_gorder, n_groups, lg;
    uint32_t off_subs, per_node, sampler, off_geo;
    uint64_t geo_full, geo_last;
    uint32_t off_wgroups;
    uint32_t stage_off;  /* byte offset in the image of the staged bytes */
    uint32_t compiled;   /* 1: the batch module holds this network's code */
    uint32_t team;       /* > 0: the team interpreter with this many warps per team of 32 lg
                            trajectories (lg per lane; nt / (32 lg) teams per item); 0: lane
                            groups of lg lanes per trajectory */
    uint32_t meta_row[PBN_BATCH_META_ROWS];
    uint32_t meta_mask[PBN_BATCH_META_ROWS];
    uint32_t meta_val[PBN_BATCH_META_ROWS];
};

struct alignas(16) pbn_workitem {
    uint32_t net, t0, n, pad;
};

struct pbn_batch_params {
    const pbn_netdesc* nets;
    const pbn_workitem* items;
    uint32_t* queue;  /* [2]: next item, CTAs done */
    uint32_t* status;
    uint64_t step_offset;
    uint32_t n_items;
    uint32_t n_steps;
};

#if defined(__CUDACC__)

/* The launch fields of one work item: its first step, the counting window of this
 * launch and the initial-state mode (the same quantities pbn_simulate computes). */
struct pbn_item_window {
    uint64_t step_begin;
    uint32_t n_steps, kv0, kp0, pairs, count_first, init;
};

__device__ __forceinline__ pbn_item_window pbn_item_window_at(const pbn_netdesc& D, uint64_t step_offset,
                                                             uint32_t n_steps) {
    pbn_item_window w;
    const uint64_t sb = D.step_begin + step_offset;
    w.step_begin = sb;
    w.n_steps = n_steps;
    /* produced states s(u) counted iff u >= count_from, pairs (s(t), s(t+1)) iff
     * t >= count_from, the initial state only when the launch starts the trajectory
     * (keyed s(0), count_from = 0): chained launches count each state once */
    const uint64_t cf = D.count_from, ns = n_steps;
    const uint64_t kv0 = cf > sb + 1 ? cf - sb - 1 : 0, kp0 = cf > sb ? cf - sb : 0;
    w.kv0 = (uint32_t)(kv0 < ns ? kv0 : ns);
    w.kp0 = (uint32_t)(kp0 < ns ? kp0 : ns);
    w.pairs = (uint32_t)(ns - w.kp0);
    w.init = (step_offset == 0) ? D.init : 1u;
    w.count_first = (w.init == 0 && cf == 0) ? 1u : 0u;
    return w;
}

/* Pooled counts of one warp: V, n00 (= pairs - the others), n01, n10, n11 summed
 * over the lanes that lead an active trajectory, one atomic per warp and count. */
__device__ __forceinline__ void pbn_warp_pool(unsigned long long* pooled, bool lead, const uint32_t c[4],
                                              uint32_t pairs) {
    uint64_t v[5] = {lead ? c[0] : 0u, lead ? (uint64_t)(pairs - c[1] - c[2] - c[3]) : 0u, lead ? c[1] : 0u,
                     lead ? c[2] : 0u, lead ? c[3] : 0u};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xFFFFFFFFu, v[i], o);
    }
    if ((threadIdx.x & 31u) == 0 && pooled) {
#pragma unroll
        for (int i = 0; i < 5; ++i)
            if (v[i]) atomicAdd(pooled + i, (unsigned long long)v[i]);
    }
}

/* The persistent loop.  `run(W, D, meta_sh, c)` simulates work item W of network D
 * (meta_sh: the network's meta rows, masks and values in shared memory) and returns
 * in c[0..3] the counts V, n01, n10, n11 of the trajectory the calling thread leads
 * (zero otherwise); it returns whether the thread leads an active trajectory. */
template <class Run>
__device__ __forceinline__ void pbn_batch_loop(const pbn_batch_params& B, uint8_t* smem, uint64_t* bar,
                                               uint32_t* item_sh, uint32_t* meta_sh, Run&& run) {
    if (threadIdx.x == 0) pbn_mbar_init(bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    uint32_t staged = 0xFFFFFFFFu;
    bool failed = false;
    for (;;) {
        if (threadIdx.x == 0) *item_sh = atomicAdd(&B.queue[0], 1u);
        __syncthreads();
        const uint32_t it = *item_sh;
        /* the previous item read and wrote shared memory through the generic proxy; the
         * bulk copies that re-stage it go through the async proxy, so every thread
         * orders its accesses before them (fence, then the barrier, then the copy) */
        pbn_fence_proxy_async();
        __syncthreads(); /* everyone has read item_sh (and finished with the previous item) */
        if (it >= B.n_items) break;
        const pbn_workitem W = B.items[it];
        const pbn_netdesc& D = B.nets[W.net];
        if (W.net != staged) {
            if (threadIdx.x == 0 && D.stage_bytes) {
                pbn_mbar_arrive_expect_tx(bar, D.stage_bytes);
                for (uint32_t off = 0; off < D.stage_bytes; off += 65536u) {
                    const uint32_t sz = (D.stage_bytes - off) < 65536u ? (D.stage_bytes - off) : 65536u;
                    pbn_bulk_g2s(smem + off, D.image + D.stage_off + off, sz, bar);
                }
            }
            if (threadIdx.x < 3 * PBN_BATCH_META_ROWS) {
                const uint32_t k = threadIdx.x;
                meta_sh[k] = k < PBN_BATCH_META_ROWS       ? D.meta_row[k]
                             : k < 2 * PBN_BATCH_META_ROWS ? D.meta_mask[k - PBN_BATCH_META_ROWS]
                                                           : D.meta_val[k - 2 * PBN_BATCH_META_ROWS];
            }
            bool ok = true;
            if (D.stage_bytes) {
                ok = false;
                for (uint32_t i = 0; i < (1u << 22); ++i) {
                    if (pbn_mbar_try_wait(bar, phase)) {
                        ok = true;
                        break;
                    }
                    if (i > 64) __nanosleep(128);
                }
            }
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            if (D.stage_bytes) phase ^= 1u;
            staged = W.net;
        }
        uint32_t c[4] = {0, 0, 0, 0};
        const bool lead = run(W, D, meta_sh, c);
        pbn_warp_pool(D.pooled, lead, c, pbn_item_window_at(D, B.step_offset, B.n_steps).pairs);
    }
    if (failed) {
        for (uint32_t i = 0; i < (1u << 22); ++i) /* let copies in flight land */
            if (pbn_mbar_try_wait(bar, phase)) break;
        if (threadIdx.x == 0 && B.status) atomicOr(B.status, PBN_BATCH_STAGE_TIMEOUT);
    }
    /* the last CTA out resets the queue for the next launch */
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&B.queue[1], 1u);
        if (done == gridDim.x - 1) {
            atomicExch(&B.queue[0], 0u);
            atomicExch(&B.queue[1], 0u);
            __threadfence();
        }
    }
}

#endif /* __CUDACC__ */
#endif /* PBN_BATCH_CUH */
