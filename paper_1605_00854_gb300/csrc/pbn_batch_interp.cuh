/*
 * pbn_batch_interp.cuh -- one work item of a batch run by the interpreter loop
 * (pbn_interp.cuh): the item's view of its network descriptor and the dispatch on
 * its lanes per trajectory and staging mode.  Used by the library's batch kernel
 * (pbn_batch.cu) and by the interpreter's work-item function that batch modules
 * link against (pbn_batch_item.cu).
 */
#ifndef PBN_BATCH_INTERP_CUH
#define PBN_BATCH_INTERP_CUH

#include "pbn_batch.cuh"
#include "pbn_interp.cuh"
#include "pbn_team.cuh"

/* The per-item view pbn_interp_run reads (the field names of the single-network
 * kernel's launch parameters). */
struct pbn_item_view {
    const uint8_t* image;
    uint64_t* state;
    uint64_t* counts;
    uint64_t* trace;
    uint64_t traj_begin, step_begin;
    uint32_t key0[10], key1[10];
    uint32_t n_traj, n_steps, kv0, kp0, pairs, count_first, init;
    uint32_t n, W, W32, n_sel, P, hmax;
    uint32_t off_words, off_groups, off_multi, off_selslot, off_thr, off_inputs, off_selblk, off_gorder, off_ret,
        off_pos, off_tables, n_groups, off_subs, per_node, sampler, off_geo, off_wgroups;
    uint64_t geo_full, geo_last;
    uint32_t n_meta_rows;
    uint32_t trace_stride;
    const uint32_t* meta_row;
    const uint32_t* meta_mask;
    const uint32_t* meta_val;
};

/* Run work item W of network D with the interpreter for n_steps steps from the
 * network's step_begin + step_offset (the network's image staged at the start of
 * smem as D's staging mode says); c[] receives the counts of the trajectory this
 * thread leads; returns whether it leads one. */
__device__ __forceinline__ bool pbn_batch_interp_run(uint64_t step_offset, uint32_t n_steps, const pbn_workitem& W,
                                                     const pbn_netdesc& D, uint8_t* smem, const uint32_t* meta_sh,
                                                     uint32_t c[4]) {
    pbn_item_view V;
    V.image = D.image;
    V.state = D.state;
    V.counts = D.counts;
    V.trace = nullptr;
    V.trace_stride = 1;
    V.traj_begin = D.traj_begin;
    const pbn_item_window w = pbn_item_window_at(D, step_offset, n_steps);
    V.step_begin = w.step_begin;
    const uint32_t k0 = (uint32_t)D.seed, k1 = (uint32_t)(D.seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        V.key0[r] = k0 + (uint32_t)r * PBN_WEYL0;
        V.key1[r] = k1 + (uint32_t)r * PBN_WEYL1;
    }
    V.n_traj = D.n_traj;
    V.n_steps = w.n_steps;
    V.kv0 = w.kv0;
    V.kp0 = w.kp0;
    V.pairs = w.pairs;
    V.count_first = w.count_first;
    V.init = w.init;
    V.n = D.n;
    V.W = D.W;
    V.W32 = D.W32;
    V.n_sel = D.n_sel;
    V.P = D.P;
    V.hmax = D.hmax;
    V.off_words = D.off_words;
    V.off_groups = D.off_groups;
    V.off_multi = D.off_multi;
    V.off_selslot = D.off_selslot;
    V.off_gorder = D.off_gorder;
    V.off_wgroups = D.off_wgroups;
    V.off_subs = D.off_subs;
    V.per_node = D.per_node;
    V.sampler = D.sampler;
    V.off_geo = D.off_geo;
    V.geo_full = D.geo_full;
    V.geo_last = D.geo_last;
    V.n_groups = D.n_groups;
    V.off_thr = D.off_thr;
    V.off_inputs = D.off_inputs;
    V.off_selblk = D.off_selblk;
    V.off_ret = D.off_ret;
    V.off_pos = D.off_pos;
    V.off_tables = D.off_tables;
    V.n_meta_rows = D.n_meta_rows;
    V.meta_row = meta_sh;
    V.meta_mask = meta_sh + PBN_BATCH_META_ROWS;
    V.meta_val = meta_sh + 2 * PBN_BATCH_META_ROWS;
    if (D.team) {
        /* teams of D.team warps on 32 x D.lg trajectories each (D.lg per lane); every
         * warp of the CTA is in one (the team count divides the CTA's warps) */
        const uint32_t K = D.team, tpl = D.lg, warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
        const uint32_t team = warp / K, wt = warp - team * K;
        const uint32_t slot0 = team * 32u * tpl + lane;
        const uint64_t lt0 = (uint64_t)W.t0 + slot0;
        uint32_t act = 0;
        for (uint32_t j = 0; j < tpl; ++j) act |= (slot0 + 32u * j < W.n ? 1u : 0u) << j;
        uint8_t* const tsm = smem + D.smem_state_off + team * pbn_team_smem_bytes(D.W32, D.n_sel, tpl);
        if (tpl == 2) {
            uint32_t c2[8];
            if (D.tables_in_smem) pbn_team_run<2, false, true>(V, smem, tsm, K, wt, lane, lt0, act, c2);
            else pbn_team_run<2, false, false>(V, smem, tsm, K, wt, lane, lt0, act, c2);
            /* the second trajectory's counts pooled here, the first one's by the caller */
            pbn_warp_pool(D.pooled, wt == 0 && ((act >> 1) & 1u), c2 + 4, V.pairs);
#pragma unroll
            for (int i = 0; i < 4; ++i) c[i] = c2[i];
        } else {
            if (D.tables_in_smem) pbn_team_run<1, false, true>(V, smem, tsm, K, wt, lane, lt0, act, c);
            else pbn_team_run<1, false, false>(V, smem, tsm, K, wt, lane, lt0, act, c);
        }
        return wt == 0 && (act & 1u);
    }
    /* D.lg lanes per trajectory, D.nt trajectory slots per item */
    const uint32_t lg = D.lg;
    const uint32_t slot = threadIdx.x / lg;
    const uint32_t lane = threadIdx.x % lg;
    const bool active = slot < W.n;
    const uint64_t lt = (uint64_t)W.t0 + slot;
    const uint32_t so = D.smem_state_off, nt = D.nt;
    if (!D.specs_in_smem) {
        pbn_interp_run<1, false, false, false>(V, smem, so, nt, slot, lane, lt, active, c);
    } else if (D.tables_in_smem) {
        switch (lg) {
            case 1: pbn_interp_run<1, false, true, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
            case 2: pbn_interp_run<2, false, true, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
            case 4: pbn_interp_run<4, false, true, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
            case 8: pbn_interp_run<8, false, true, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
            case 16: pbn_interp_run<16, false, true, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
            default: pbn_interp_run<32, false, true, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
        }
    } else {
        switch (lg) {
            case 1: pbn_interp_run<1, false, false, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
            case 2: pbn_interp_run<2, false, false, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
            case 4: pbn_interp_run<4, false, false, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
            case 8: pbn_interp_run<8, false, false, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
            case 16: pbn_interp_run<16, false, false, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
            default: pbn_interp_run<32, false, false, true>(V, smem, so, nt, slot, lane, lt, active, c); break;
        }
    }
    return active && lane == 0;
}

/* Body of the library's interpreted batch kernels (one per CTA size). */
__device__ __forceinline__ void pbn_batch_interp_kernel_body(const pbn_batch_params& B) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t item_sh;
    __shared__ uint32_t meta_sh[3 * PBN_BATCH_META_ROWS];
    pbn_batch_loop(B, smem, &bar, &item_sh, meta_sh,
                   [&](const pbn_workitem& W, const pbn_netdesc& D, const uint32_t* ms, uint32_t c[4]) -> bool {
                       return pbn_batch_interp_run(B.step_offset, B.n_steps, W, D, smem, ms, c);
                   });
}

#endif /* PBN_BATCH_INTERP_CUH */
