/*
 * pbn_batch.cu -- many networks in one persistent launch fed by a device work
 * queue (the batched form of Algorithm 5's ParallelSimulation).
 *
 * Host side (pbn_batch_create): every network is cut into work items of up to
 * `blockDim` trajectories; the items are ordered by descending estimated cost
 * (largest processing time first) so that the persistent CTAs finish together.
 * The per-network descriptors (plan image pointer, plan offsets, Philox seed,
 * counting window, meta-state rows, output pointers) and the item list form one
 * device table the caller uploads (pbn_batch_image).
 *
 * Device side (pbn_batch_kernel): a grid of SMs x k CTAs; each CTA pops the next
 * item with one atomic, bulk-copies the item's plan image into shared memory when
 * it differs from the one it holds (cp.async.bulk + mbarrier, bounded wait), runs
 * the interpreter loop for `n_steps` steps on the item's trajectories and pools
 * its counts.  A launch advances every network by n_steps steps from
 * step_begin + step_offset, so a long run is a chain of launches (one chunk each)
 * that the caller can capture in a CUDA graph.  The queue is two uint32 counters
 * in caller memory: the next item and the number of CTAs that found the queue
 * empty; the last CTA to leave resets both to zero, so consecutive launches need
 * no host reset.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "pbn_device.cuh"
#include "pbn_interp.cuh"
#include "pbn_internal.h"

namespace {

constexpr uint32_t kWeyl0 = 0x9E3779B9u;
constexpr uint32_t kWeyl1 = 0xBB67AE85u;
constexpr uint32_t kMetaRows = 16;
constexpr uint64_t kSmemCap = 224u * 1024u; /* per-CTA shared memory: one 512-thread CTA per SM, so
                                                 the specs of every network fit in shared memory */

/* Per-network descriptor in device memory (written by the host, read-only). */
struct alignas(16) NetDesc {
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
    uint32_t off_wgroups, pad0, pad1, pad2;
    uint32_t meta_row[kMetaRows];
    uint32_t meta_mask[kMetaRows];
    uint32_t meta_val[kMetaRows];
};

struct alignas(16) WorkItem {
    uint32_t net, t0, n, pad;
};

struct BatchParams {
    const NetDesc* nets;
    const WorkItem* items;
    uint32_t* queue;     /* [2]: next item, CTAs done */
    uint32_t* status;
    uint64_t step_offset;
    uint32_t n_items;
    uint32_t n_steps;
};

/* The per-item view pbn_interp_run reads (same field names as the launch
 * parameters of the single-network kernel). */
struct ItemView {
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

__device__ __forceinline__ void warp_pool(unsigned long long* pooled, bool lead, const uint32_t c[4], uint32_t pairs) {
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

__global__ void __launch_bounds__(512, 1) pbn_batch_kernel(const BatchParams B) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t item_sh;
    __shared__ uint32_t meta_sh[3 * kMetaRows];
    if (threadIdx.x == 0) pbn_mbar_init(&bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    uint32_t staged = 0xFFFFFFFFu;
    bool failed = false;
    for (;;) {
        if (threadIdx.x == 0) item_sh = atomicAdd(&B.queue[0], 1u);
        __syncthreads();
        const uint32_t it = item_sh;
        /* the previous item read and wrote shared memory through the generic proxy; the
         * bulk copies that re-stage it go through the async proxy, so every thread
         * orders its accesses before them (fence, then the barrier, then the copy) */
        pbn_fence_proxy_async();
        __syncthreads(); /* everyone has read item_sh (and finished with the previous plan) */
        if (it >= B.n_items) break;
        const WorkItem W = B.items[it];
        const NetDesc& D = B.nets[W.net];
        if (W.net != staged) {
            if (threadIdx.x == 0 && D.stage_bytes) {
                pbn_mbar_arrive_expect_tx(&bar, D.stage_bytes);
                for (uint32_t off = 0; off < D.stage_bytes; off += 65536u) {
                    const uint32_t sz = (D.stage_bytes - off) < 65536u ? (D.stage_bytes - off) : 65536u;
                    pbn_bulk_g2s(smem + off, D.image + off, sz, &bar);
                }
            }
            if (threadIdx.x < 3 * kMetaRows) {
                const uint32_t k = threadIdx.x;
                meta_sh[k] = k < kMetaRows ? D.meta_row[k] : (k < 2 * kMetaRows ? D.meta_mask[k - kMetaRows]
                                                                                  : D.meta_val[k - 2 * kMetaRows]);
            }
            bool ok = true;
            if (D.stage_bytes) {
                ok = false;
                for (uint32_t i = 0; i < (1u << 22); ++i) {
                    if (pbn_mbar_try_wait(&bar, phase)) { ok = true; break; }
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
        /* the view of this item */
        ItemView V;
        V.image = D.image;
        V.state = D.state;
        V.counts = D.counts;
        V.trace = nullptr;
        V.trace_stride = 1;
        V.traj_begin = D.traj_begin;
        const uint64_t sb = D.step_begin + B.step_offset;
        V.step_begin = sb;
        const uint32_t k0 = (uint32_t)D.seed, k1 = (uint32_t)(D.seed >> 32);
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            V.key0[r] = k0 + (uint32_t)r * kWeyl0;
            V.key1[r] = k1 + (uint32_t)r * kWeyl1;
        }
        V.n_traj = D.n_traj;
        V.n_steps = B.n_steps;
        const uint64_t cf = D.count_from, ns = B.n_steps;
        const uint64_t kv0 = cf > sb + 1 ? cf - sb - 1 : 0, kp0 = cf > sb ? cf - sb : 0;
        V.kv0 = (uint32_t)(kv0 < ns ? kv0 : ns);
        V.kp0 = (uint32_t)(kp0 < ns ? kp0 : ns);
        V.pairs = (uint32_t)(ns - V.kp0);
        V.count_first = sb == cf ? 1u : 0u;
        V.init = (B.step_offset == 0) ? D.init : 1u;
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
        V.meta_mask = meta_sh + kMetaRows;
        V.meta_val = meta_sh + 2 * kMetaRows;
        /* D.lg lanes per trajectory, D.nt trajectory slots per item */
        const uint32_t lg = D.lg;
        const uint32_t slot = threadIdx.x / lg;
        const uint32_t lane = threadIdx.x % lg;
        const bool active = slot < W.n;
        const uint64_t lt = (uint64_t)W.t0 + slot;
        uint32_t c[4] = {0, 0, 0, 0};
        if (!D.specs_in_smem) {
            pbn_interp_run<1, false, false, false>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c);
        } else if (D.tables_in_smem) {
            switch (lg) {
                case 1: pbn_interp_run<1, false, true, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
                case 2: pbn_interp_run<2, false, true, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
                case 4: pbn_interp_run<4, false, true, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
                case 8: pbn_interp_run<8, false, true, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
                case 16: pbn_interp_run<16, false, true, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
                default: pbn_interp_run<32, false, true, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
            }
        } else {
            switch (lg) {
                case 1: pbn_interp_run<1, false, false, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
                case 2: pbn_interp_run<2, false, false, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
                case 4: pbn_interp_run<4, false, false, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
                case 8: pbn_interp_run<8, false, false, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
                case 16: pbn_interp_run<16, false, false, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
                default: pbn_interp_run<32, false, false, true>(V, smem, D.smem_state_off, D.nt, slot, lane, lt, active, c); break;
            }
        }
        warp_pool(D.pooled, active && lane == 0, c, V.pairs);
    }
    if (failed) {
        for (uint32_t i = 0; i < (1u << 22); ++i) /* let copies in flight land */
            if (pbn_mbar_try_wait(&bar, phase)) break;
        if (threadIdx.x == 0 && B.status) atomicOr(B.status, PBN_DEV_STAGE_TIMEOUT);
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

constexpr int kMaxDevices = 64;

}  // namespace

struct pbn_batch {
    pbn_batch_info info{};
    std::vector<NetDesc> nets;
    std::vector<WorkItem> items;
    std::vector<uint8_t> image; /* nets then items */
    uint32_t threads = 512;
    /* CTAs of the batch kernel per SM and the SM count, per device, found on the first
     * run on that device (so that later launches can be graph-captured) */
    mutable std::mutex mu;
    mutable int occ_per_sm[kMaxDevices] = {0};
    mutable int sms[kMaxDevices] = {0};
};

namespace {

/* Meta-state rows of network i: per 32-bit state row holding a meta node, the mask
 * of those nodes and the values they must take. */
int describe_meta(const pbn_batch_net& a, uint32_t i, NetDesc* D) {
    using pbn::fail;
    if (a.n_meta < 1 || a.n_meta > 1024 || !a.meta_ids)
        return fail(PBN_EINVAL, "pbn_batch_create: network %u needs 1..1024 meta nodes", i);
    char who[64];
    snprintf(who, sizeof who, "pbn_batch_create: network %u", i);
    pbn::MetaRows M;
    const int rc = pbn::meta_rows(a.plan, a.meta_ids, a.meta_vals, a.n_meta, kMetaRows, who, &M);
    if (rc != PBN_OK) return rc;
    D->n_meta_rows = M.n_rows;
    for (uint32_t k = 0; k < M.n_rows; ++k) {
        D->meta_row[k] = M.row[k];
        D->meta_mask[k] = M.mask[k];
        D->meta_val[k] = M.val[k];
    }
    return PBN_OK;
}

/* Descriptor of network i for a CTA of T threads: buffers, counting window, meta
 * rows, image section offsets, and the staging mode with its trajectory slots per
 * work item and lanes per trajectory. */
int describe_network(const pbn_batch_net& a, uint32_t i, uint32_t T, NetDesc* D) {
    using pbn::fail;
    const pbn_plan* plan = a.plan;
    if (!plan || !a.d_image || ((uintptr_t)a.d_image & 15u) || !a.d_state)
        return fail(PBN_EINVAL, "pbn_batch_create: network %u lacks a plan, image or state", i);
    if (a.n_traj == 0 || a.n_traj >= (1ull << 31) || a.traj_begin + a.n_traj > (1ull << 48))
        return fail(PBN_EINVAL, "pbn_batch_create: network %u trajectory range", i);
    if (a.init != PBN_INIT_KEYED && a.init != PBN_INIT_STATE)
        return fail(PBN_EINVAL, "pbn_batch_create: network %u init mode", i);
    if (a.init == PBN_INIT_KEYED && a.step_begin != 0)
        return fail(PBN_EINVAL, "pbn_batch_create: network %u keyed init needs step_begin 0", i);
    const pbn_img_header& H = plan->hdr;
    memset(D, 0, sizeof(*D));
    const int rc = describe_meta(a, i, D);
    if (rc != PBN_OK) return rc;
    D->image = static_cast<const uint8_t*>(a.d_image);
    D->state = static_cast<uint64_t*>(a.d_state);
    D->counts = static_cast<uint64_t*>(a.d_counts);
    D->pooled = static_cast<unsigned long long*>(a.d_pooled);
    D->traj_begin = a.traj_begin;
    D->step_begin = a.step_begin;
    D->count_from = a.count_from;
    D->seed = a.seed;
    D->n_traj = (uint32_t)a.n_traj;
    D->init = a.init;
    D->image_bytes = H.image_bytes;
    D->hmax = H.P ? (31u - (uint32_t)__builtin_ctz(H.P)) / 2u + 1u : 0u;
    D->n = H.n;
    D->W = H.W;
    D->W32 = H.W32;
    D->n_sel = H.n_sel;
    D->P = H.P;
    D->off_words = H.off_words;
    D->off_groups = H.off_groups;
    D->off_multi = H.off_multi;
    D->off_selslot = H.off_selslot;
    D->off_gorder = H.off_gorder;
    D->off_wgroups = H.off_wgroups;
    D->off_subs = H.off_subs;
    D->per_node = H.semantics == PBN_SEM_NODEWISE ? 1u : 0u;
    D->sampler = H.sampler;
    D->off_geo = H.off_geo;
    {
        const uint64_t* G = reinterpret_cast<const uint64_t*>(plan->image.data() + H.off_geo);
        const uint32_t nl = H.n & 63u;
        D->geo_full = G[63];
        D->geo_last = G[(nl ? nl : 64u) - 1];
    }
    D->n_groups = H.n_groups;
    D->off_thr = H.off_thr;
    D->off_inputs = H.off_inputs;
    D->off_selblk = H.off_selblk;
    D->off_ret = H.off_ret;
    D->off_pos = H.off_pos;
    D->off_tables = H.off_tables;
    /* staging mode and trajectories per work item under the per-CTA cap:
     * specs and tables staged, specs only, or nothing (read through L1) */
    const uint64_t per = plan->per_traj_smem;
    auto fit = [&](uint64_t staged) -> uint32_t {
        const uint64_t off = (staged + 127u) & ~(uint64_t)127u;
        if (off + per * 32 > kSmemCap) return 0u;
        uint64_t nt = (kSmemCap - off) / per;
        nt = std::min<uint64_t>(T, nt & ~(uint64_t)31);
        return (uint32_t)nt;
    };
    const uint32_t nt_all = H.tables_in_smem ? fit(H.off_ret) : 0u;
    const uint32_t nt_specs = fit(H.off_tables);
    const uint32_t nt_none = fit(0);
    if (nt_all >= std::min<uint32_t>(T, 256u) || (nt_all && nt_all >= nt_specs)) {
        D->specs_in_smem = 1; D->tables_in_smem = 1; D->stage_bytes = H.off_ret; D->nt = nt_all;
    } else if (nt_specs) {
        D->specs_in_smem = 1; D->tables_in_smem = 0; D->stage_bytes = H.off_tables; D->nt = nt_specs;
    } else if (nt_none) {
        D->specs_in_smem = 0; D->tables_in_smem = 0; D->stage_bytes = 0; D->nt = nt_none;
    } else {
        return fail(PBN_ETOOBIG, "pbn_batch_create: network %u needs %llu bytes of shared memory per trajectory", i,
                    (unsigned long long)per);
    }
    D->smem_state_off = D->stage_bytes ? ((D->stage_bytes + 127u) & ~127u) : 0u;
    /* lanes per trajectory: fill the CTA's threads when few trajectories fit (wide
     * states); lane groups evaluate groups in shape order.  States of 32 words or more
     * take up to a warp per trajectory (two words per lane: 32 lanes ran a 62-word
     * state 1.66x faster than 8), smaller ones up to 8 lanes with at least 8 words each */
    D->lg = 1;
    if (D->specs_in_smem) {
        const bool wide_state = D->W32 >= 32;
        const uint32_t lg_max = wide_state ? 32u : 8u, words_per_lane = wide_state ? 2u : 8u;
        while (D->lg < lg_max && D->nt * D->lg * 2 <= T && D->W32 >= words_per_lane * D->lg) D->lg *= 2;
    }
    return PBN_OK;
}

}  // namespace

extern "C" int pbn_batch_create(const pbn_batch_net* nets, uint32_t n_nets, pbn_batch** out) {
    using pbn::fail;
    if (!nets || !out || n_nets == 0) return fail(PBN_EINVAL, "pbn_batch_create: need networks");
    *out = nullptr;
    try {
        std::unique_ptr<pbn_batch> B(new pbn_batch());
        const uint32_t T = B->threads;
        uint64_t smem_max = 0;
        uint32_t max_lanes = 1;
        std::vector<double> cost_per_traj(n_nets);
        for (uint32_t i = 0; i < n_nets; ++i) {
            const pbn_batch_net& a = nets[i];
            NetDesc D;
            const int rc = describe_network(a, i, T, &D);
            if (rc != PBN_OK) return rc;
            max_lanes = std::max(max_lanes, D.lg);
            smem_max = std::max<uint64_t>(smem_max, D.smem_state_off + (uint64_t)a.plan->per_traj_smem * D.nt);
            cost_per_traj[i] = a.plan->info.ops_per_step;
            B->nets.push_back(D);
            for (uint64_t t0 = 0; t0 < a.n_traj; t0 += D.nt) {
                WorkItem w{i, (uint32_t)t0, (uint32_t)std::min<uint64_t>(D.nt, a.n_traj - t0), 0u};
                B->items.push_back(w);
            }
        }
        /* largest estimated work first */
        std::stable_sort(B->items.begin(), B->items.end(), [&](const WorkItem& x, const WorkItem& y) {
            return cost_per_traj[x.net] * x.n > cost_per_traj[y.net] * y.n;
        });
        B->info.n_nets = n_nets;
        B->info.n_items = (uint32_t)B->items.size();
        B->info.smem_bytes = smem_max;
        B->info.threads = T;
        B->info.max_lanes = max_lanes;
        double ops = 0;
        for (uint32_t i = 0; i < n_nets; ++i) ops += cost_per_traj[i] * (double)nets[i].n_traj;
        B->info.est_ops_per_step = ops;
        const size_t nb = B->nets.size() * sizeof(NetDesc), ib = B->items.size() * sizeof(WorkItem);
        B->image.resize(nb + ib);
        memcpy(B->image.data(), B->nets.data(), nb);
        memcpy(B->image.data() + nb, B->items.data(), ib);
        B->info.desc_bytes = B->image.size();
        *out = B.release();
        return PBN_OK;
    } catch (const std::bad_alloc&) {
        return fail(PBN_ENOMEM, "pbn_batch_create: out of memory");
    }
}

extern "C" void pbn_batch_free(pbn_batch* b) { delete b; }

extern "C" int pbn_batch_info_get(const pbn_batch* b, pbn_batch_info* out) {
    if (!b || !out) return pbn::fail(PBN_EINVAL, "pbn_batch_info_get: NULL argument");
    *out = b->info;
    return PBN_OK;
}

extern "C" int pbn_batch_image(const pbn_batch* b, void* dst, size_t cap) {
    if (!b || !dst) return pbn::fail(PBN_EINVAL, "pbn_batch_image: NULL argument");
    if (cap < b->image.size()) return pbn::fail(PBN_EINVAL, "pbn_batch_image: need %zu bytes", b->image.size());
    memcpy(dst, b->image.data(), b->image.size());
    return PBN_OK;
}

namespace {
/* Grid of the batch kernel on the current device: raises the kernel's shared-memory
 * limit there to the batch's need (never lowering what another batch set), and finds
 * the CTAs per SM and the SM count of that device on the batch's first run on it. */
int launch_shape(const pbn_batch* b, uint32_t ctas_per_sm, const char* who, uint32_t* grid) {
    using pbn::fail;
    const size_t smem = b->info.smem_bytes;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PBN_ECUDA, "%s: %s", who, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PBN_EINVAL, "%s: device %d beyond %d", who, dev, kMaxDevices);
    const int se = pbn::ensure_dyn_smem(reinterpret_cast<const void*>(pbn_batch_kernel), smem);
    if (se != 0) return fail(PBN_ECUDA, "%s: %s", who, cudaGetErrorString(static_cast<cudaError_t>(se)));
    int per_sm = 0, sms = 0;
    {
        std::lock_guard<std::mutex> g(b->mu);
        if (!b->occ_per_sm[dev]) {
            int occ = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pbn_batch_kernel, (int)b->threads, smem);
            if (e != cudaSuccess || occ < 1) return fail(PBN_ETOOBIG, "%s: the batch kernel does not fit an SM", who);
            b->occ_per_sm[dev] = occ;
            b->sms[dev] = pbn::device_sms();
        }
        per_sm = b->occ_per_sm[dev];
        sms = b->sms[dev];
    }
    if (ctas_per_sm && (int)ctas_per_sm < per_sm) per_sm = (int)ctas_per_sm;
    *grid = (uint32_t)std::min<uint64_t>((uint64_t)sms * per_sm, std::max<uint32_t>(1u, b->info.n_items));
    return PBN_OK;
}
}  // namespace

extern "C" int pbn_batch_run(const pbn_batch* b, const void* d_desc, uint32_t* d_queue, uint64_t step_offset,
                             uint64_t n_steps, uint32_t ctas_per_sm, uint32_t* d_status, void* stream) {
    using pbn::fail;
    if (!b || !d_desc || !d_queue) return fail(PBN_EINVAL, "pbn_batch_run: NULL argument");
    if (((uintptr_t)d_desc & 15u) || ((uintptr_t)d_queue & 3u)) return fail(PBN_EINVAL, "pbn_batch_run: misaligned buffer");
    if (n_steps >= (1ull << 32)) return fail(PBN_EINVAL, "pbn_batch_run: n_steps must be < 2^32");
    for (const NetDesc& D : b->nets)
        if (D.step_begin + step_offset + n_steps > (1ull << 48)) return fail(PBN_EINVAL, "pbn_batch_run: step index >= 2^48");
    BatchParams P;
    P.nets = static_cast<const NetDesc*>(d_desc);
    P.items = reinterpret_cast<const WorkItem*>(static_cast<const uint8_t*>(d_desc) + b->nets.size() * sizeof(NetDesc));
    P.queue = d_queue;
    P.status = d_status;
    P.step_offset = step_offset;
    P.n_items = b->info.n_items;
    P.n_steps = (uint32_t)n_steps;
    const size_t smem = b->info.smem_bytes;
    uint32_t grid = 0;
    int rc = launch_shape(b, ctas_per_sm, "pbn_batch_run", &grid);
    if (rc != PBN_OK) return rc;
    pbn_batch_kernel<<<grid, b->threads, smem, static_cast<cudaStream_t>(stream)>>>(P);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PBN_ECUDA, "pbn_batch_run: %s", cudaGetErrorString(e));
    return PBN_OK;
}

/* ---- allocation-free variant of pbn_batch_run ------------------------------------------
 * Some callers cannot allocate device memory at the point where they run a batch: a
 * serving loop or an embedding framework whose allocator owns the whole device, code
 * that records its launches into a CUDA graph (allocation is not allowed during stream
 * capture), and latency-critical loops that must not call cudaMalloc or cudaFree,
 * which can synchronise the whole device.  This entry point takes the work-queue
 * scratch from a small array the library owns in device memory instead of from the
 * caller.  The array has PBN_STATIC_QUEUE_SLOTS independent queues of two counters
 * (128 bytes in all); every GPU that loads the library keeps it until the process
 * exits. */
namespace {
__device__ __align__(256) uint32_t g_pbn_static_queues[2 * PBN_STATIC_QUEUE_SLOTS];

std::mutex g_static_mu;
uint32_t* g_static_addr[kMaxDevices] = {nullptr};
}  // namespace

extern "C" int pbn_batch_run_static(const pbn_batch* b, const void* d_desc, uint32_t slot, uint64_t step_offset,
                                    uint64_t n_steps, uint32_t ctas_per_sm, uint32_t* d_status, void* stream) {
    using pbn::fail;
    if (!b || !d_desc) return fail(PBN_EINVAL, "pbn_batch_run_static: NULL argument");
    if (slot >= PBN_STATIC_QUEUE_SLOTS)
        return fail(PBN_EINVAL, "pbn_batch_run_static: queue slot %u is beyond the library's %u static slots", slot,
                    (unsigned)PBN_STATIC_QUEUE_SLOTS);
    if ((uintptr_t)d_desc & 15u) return fail(PBN_EINVAL, "pbn_batch_run_static: misaligned descriptor table");
    if (n_steps >= (1ull << 32)) return fail(PBN_EINVAL, "pbn_batch_run_static: n_steps must be < 2^32");
    for (const NetDesc& D : b->nets)
        if (D.step_begin + step_offset + n_steps > (1ull << 48))
            return fail(PBN_EINVAL, "pbn_batch_run_static: step index >= 2^48");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PBN_ECUDA, "pbn_batch_run_static: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PBN_EINVAL, "pbn_batch_run_static: device %d beyond %d", dev, kMaxDevices);
    uint32_t* base = nullptr;
    {
        /* once per device, with that device current: the host-side name of the array
         * is not a device address, so ask the runtime for the address */
        std::lock_guard<std::mutex> g(g_static_mu);
        if (!g_static_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_pbn_static_queues);
            if (e != cudaSuccess || !p)
                return fail(PBN_ECUDA, "pbn_batch_run_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_static_addr[dev] = static_cast<uint32_t*>(p);
        }
        base = g_static_addr[dev];
    }
    uint32_t* q = base + 2 * slot;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    /* the array keeps the last call's counters: start this launch's queue at zero */
    e = cudaMemsetAsync(q, 0, 2 * sizeof(uint32_t), st);
    if (e != cudaSuccess) return fail(PBN_ECUDA, "pbn_batch_run_static: %s", cudaGetErrorString(e));
    BatchParams P;
    P.nets = static_cast<const NetDesc*>(d_desc);
    P.items = reinterpret_cast<const WorkItem*>(static_cast<const uint8_t*>(d_desc) + b->nets.size() * sizeof(NetDesc));
    P.queue = q;
    P.status = d_status;
    P.step_offset = step_offset;
    P.n_items = b->info.n_items;
    P.n_steps = (uint32_t)n_steps;
    const size_t smem = b->info.smem_bytes;
    uint32_t grid = 0;
    const int rc = launch_shape(b, ctas_per_sm, "pbn_batch_run_static", &grid);
    if (rc != PBN_OK) return rc;
    pbn_batch_kernel<<<grid, b->threads, smem, st>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PBN_ECUDA, "pbn_batch_run_static: %s", cudaGetErrorString(e));
    return PBN_OK;
}
