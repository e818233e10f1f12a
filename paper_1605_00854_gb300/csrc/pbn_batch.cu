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
#include <string>
#include <vector>

#include "pbn_batch_interp.cuh"
#include "pbn_internal.h"

namespace {

constexpr uint32_t kMetaRows = PBN_BATCH_META_ROWS;
constexpr uint64_t kSmemCap = 224u * 1024u; /* per-CTA shared memory: one 512-thread CTA per SM, so
                                                 the specs of every network fit in shared memory */
constexpr int kMaxDevices = 64;

using NetDesc = pbn_netdesc;
using WorkItem = pbn_workitem;
using BatchParams = pbn_batch_params;

/* The batch kernel of the library: every work item runs the interpreter (CTAs of
 * 512 threads; the 1,024-thread instantiation is in pbn_batch1024.cu). */
__global__ void __launch_bounds__(512, 1) pbn_batch_kernel(const BatchParams B) { pbn_batch_interp_kernel_body(B); }

}  // namespace

namespace pbn {
const void* batch_kernel_1024();
}

struct pbn_batch {
    pbn_batch_info info{};
    std::vector<NetDesc> nets;
    std::vector<WorkItem> items;
    std::vector<uint8_t> image; /* nets then items */
    std::vector<const pbn_plan*> plans;
    uint32_t threads = 512;
    bool lane_groups = false; /* PBN_BATCH_LANE_GROUPS: no team interpreter */
    /* batch module (pbn_batch_compile): compiled networks' functions and the
     * dispatching persistent kernel, or null (the library's interpreter kernel) */
    void* module = nullptr;
    void* module_kernel = nullptr;
    /* split batch: the module runs the compiled networks' items (the first n_items_c),
     * then the library's 1,024-thread interpreter kernel the others, in a second
     * launch on the same queue */
    bool split = false;
    uint32_t n_items_c = 0;
    size_t smem_c = 0, smem_i = 0;
    mutable int occ_i[kMaxDevices] = {0};
    ~pbn_batch() { pbn::jit_library_unload(module); }
    /* CTAs of the batch kernel per SM and the SM count, per device, found on the first
     * run on that device (so that later launches can be graph-captured) */
    mutable std::mutex mu;
    mutable int occ_per_sm[kMaxDevices] = {0};
    mutable int sms[kMaxDevices] = {0};
};

namespace {

int interp_shape(const pbn_plan* plan, uint32_t T, bool teams_ok, NetDesc* D);

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
int describe_network(const pbn_batch_net& a, uint32_t i, uint32_t T, bool teams_ok, NetDesc* D) {
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
    const int rc2 = interp_shape(plan, T, teams_ok, D);
    if (rc2 != PBN_OK)
        return fail(PBN_ETOOBIG, "pbn_batch_create: network %u needs %llu bytes of shared memory per trajectory", i,
                    (unsigned long long)plan->per_traj_smem);
    return PBN_OK;
}

/* The interpreter's shape of a network's work items for CTAs of T threads: staging
 * mode and trajectory slots per item under the per-CTA shared-memory cap (specs and
 * tables staged, specs only, or nothing: read through L1), the offset of the
 * trajectory rows, and the lanes per trajectory.  PBN_ETOOBIG if not even 32
 * trajectory rows fit. */
int interp_shape(const pbn_plan* plan, uint32_t T, bool teams_ok, NetDesc* D) {
    const pbn_img_header& H = plan->hdr;
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
        return PBN_ETOOBIG;
    }
    D->stage_off = 0;
    D->compiled = 0;
    D->team = 0;
    D->smem_state_off = D->stage_bytes ? ((D->stage_bytes + 127u) & ~127u) : 0u;
    /* states of 8 rows or more (Eq. 1 semantics): the team interpreter, its records
     * staged (tables too when at least as many teams fit), two trajectories per lane
     * when such a team fits (one record decode serves both), as many teams as the
     * shared memory holds up to a power of two dividing the CTA's warps, and the
     * warps split evenly over them (on paper-scale networks of 300 to 3,000 nodes
     * and the 2,000-node scale-free one it ran 1.2-1.33x the lane groups) */
    if (teams_ok && H.W32 >= 8 && H.semantics != PBN_SEM_NODEWISE) {
        const uint32_t warps = T / 32u;
        auto teams = [&](uint64_t staged, uint32_t tpl) -> uint32_t {
            const uint64_t tb = pbn_team_smem_bytes(H.W32, H.n_sel, tpl);
            const uint64_t off = (staged + 127u) & ~(uint64_t)127u;
            if (off + tb > kSmemCap) return 0u;
            uint32_t t = 1;
            while (2 * t <= warps && off + 2 * t * tb <= kSmemCap) t *= 2;
            return t;
        };
        for (uint32_t tpl = 2; tpl >= 1; --tpl) {
            const uint32_t t_all = H.tables_in_smem ? teams(H.off_ret, tpl) : 0u;
            const uint32_t t_specs = teams(H.off_tables, tpl);
            if (!t_all && !t_specs) continue;
            if (t_all && t_all >= t_specs) {
                D->specs_in_smem = 1; D->tables_in_smem = 1; D->stage_bytes = H.off_ret; D->nt = 32u * tpl * t_all;
            } else {
                D->specs_in_smem = 1; D->tables_in_smem = 0; D->stage_bytes = H.off_tables; D->nt = 32u * tpl * t_specs;
            }
            D->team = warps / (D->nt / (32u * tpl));
            D->lg = tpl;
            D->smem_state_off = (D->stage_bytes + 127u) & ~127u;
            return PBN_OK;
        }
    }
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

namespace {
/* Interpreted work is costed at this many times a compiled network's per trajectory
 * and step when the items are ordered (the interpreter ran the paper-scale plan
 * about 3.6x slower than its compiled kernel). */
constexpr double kInterpCost = 3.0;
/* Compiled networks per batch module.  nvJitLink (CUDA 13.0) crashed the process
 * linking a dispatcher with 136 network functions (102 linked), so a module takes
 * at most this many, the networks with the most estimated work; the others run the
 * interpreter in the same launch. */
constexpr size_t kMaxCompiledNets = 96;

/* Shared memory of an interpreted network's work item: its staged bytes and the
 * trajectories' rows (lane groups) or the teams' states (team interpreter). */
uint64_t interp_smem(const NetDesc& D, const pbn_plan* plan) {
    if (D.team) return D.smem_state_off + (uint64_t)(D.nt / (32u * D.lg)) * pbn_team_smem_bytes(D.W32, D.n_sel, D.lg);
    return D.smem_state_off + (uint64_t)plan->per_traj_smem * D.nt;
}

/* Cut every network into work items of its descriptor's trajectory slots, order them
 * by descending estimated work (largest processing time first, so that the
 * persistent CTAs finish together) and lay out the device table. */
void cut_items(pbn_batch* B) {
    const uint32_t n_nets = (uint32_t)B->nets.size();
    std::vector<double> cost(n_nets);
    uint64_t smem_max = 0;
    uint32_t max_lanes = 1, n_compiled = 0, n_team = 0;
    double ops = 0;
    B->items.clear();
    for (uint32_t i = 0; i < n_nets; ++i) {
        const NetDesc& D = B->nets[i];
        const pbn_plan* plan = B->plans[i];
        cost[i] = plan->info.ops_per_step * (D.compiled ? 1.0 : kInterpCost);
        ops += plan->info.ops_per_step * (double)D.n_traj;
        if (D.compiled) {
            ++n_compiled;
            smem_max = std::max<uint64_t>(smem_max, D.stage_bytes);
        } else {
            max_lanes = std::max(max_lanes, D.team ? 32u : D.lg);
            if (D.team) ++n_team;
            smem_max = std::max<uint64_t>(smem_max, interp_smem(D, plan));
        }
        for (uint64_t t0 = 0; t0 < D.n_traj; t0 += D.nt) {
            WorkItem w{i, (uint32_t)t0, (uint32_t)std::min<uint64_t>(D.nt, D.n_traj - t0), 0u};
            B->items.push_back(w);
        }
    }
    std::stable_sort(B->items.begin(), B->items.end(), [&](const WorkItem& x, const WorkItem& y) {
        if (B->split && B->nets[x.net].compiled != B->nets[y.net].compiled) return B->nets[x.net].compiled > 0;
        return cost[x.net] * x.n > cost[y.net] * y.n;
    });
    B->n_items_c = 0;
    B->smem_c = B->smem_i = 0;
    for (const WorkItem& w : B->items)
        if (B->nets[w.net].compiled) ++B->n_items_c;
    for (uint32_t i = 0; i < n_nets; ++i) {
        const NetDesc& D = B->nets[i];
        if (D.compiled) B->smem_c = std::max<size_t>(B->smem_c, D.stage_bytes);
        else B->smem_i = std::max<size_t>(B->smem_i, interp_smem(D, B->plans[i]));
    }
    B->info.n_nets = n_nets;
    B->info.n_items = (uint32_t)B->items.size();
    B->info.smem_bytes = smem_max;
    B->info.threads = B->threads;
    B->info.max_lanes = max_lanes;
    B->info.est_ops_per_step = ops;
    B->info.n_compiled = n_compiled;
    B->info.n_team = n_team;
    B->info.n_items_compiled = B->split ? B->n_items_c : 0u;
    const size_t nb = B->nets.size() * sizeof(NetDesc), ib = B->items.size() * sizeof(WorkItem);
    B->image.resize(nb + ib);
    memcpy(B->image.data(), B->nets.data(), nb);
    memcpy(B->image.data() + nb, B->items.data(), ib);
    B->info.desc_bytes = B->image.size();
}
}  // namespace

extern "C" int pbn_batch_create(const pbn_batch_net* nets, uint32_t n_nets, pbn_batch** out) {
    return pbn_batch_create_cta(nets, n_nets, 512, out);
}

extern "C" int pbn_batch_create_cta(const pbn_batch_net* nets, uint32_t n_nets, uint32_t threads, pbn_batch** out) {
    return pbn_batch_create_ex(nets, n_nets, threads, 0u, out);
}

extern "C" int pbn_batch_create_ex(const pbn_batch_net* nets, uint32_t n_nets, uint32_t threads, uint32_t flags,
                                   pbn_batch** out) {
    using pbn::fail;
    if (!nets || !out || n_nets == 0) return fail(PBN_EINVAL, "pbn_batch_create: need networks");
    if (threads != 512 && threads != 1024) return fail(PBN_EINVAL, "pbn_batch_create: CTAs of 512 or 1024 threads");
    if (flags & ~PBN_BATCH_LANE_GROUPS) return fail(PBN_EINVAL, "pbn_batch_create: unknown flags 0x%x", flags);
    *out = nullptr;
    try {
        std::unique_ptr<pbn_batch> B(new pbn_batch());
        B->threads = threads;
        B->lane_groups = (flags & PBN_BATCH_LANE_GROUPS) != 0;
        const uint32_t T = B->threads;
        for (uint32_t i = 0; i < n_nets; ++i) {
            const pbn_batch_net& a = nets[i];
            NetDesc D;
            const int rc = describe_network(a, i, T, !B->lane_groups, &D);
            if (rc != PBN_OK) return rc;
            B->nets.push_back(D);
            B->plans.push_back(a.plan);
        }
        cut_items(B.get());
        *out = B.release();
        return PBN_OK;
    } catch (const std::bad_alloc&) {
        return fail(PBN_ENOMEM, "pbn_batch_create: out of memory");
    }
}

extern "C" int pbn_batch_compile(pbn_batch* b, uint32_t flags, double* compile_ms) {
    using pbn::fail;
    if (!b) return fail(PBN_EINVAL, "pbn_batch_compile: NULL batch");
    if (b->module) return fail(PBN_EINVAL, "pbn_batch_compile: the batch is compiled already");
    if (b->threads != 512) return fail(PBN_EINVAL, "pbn_batch_compile: compiled batches run CTAs of 512 threads");
    const bool split = (flags & PBN_BATCH_SPLIT) != 0;
    flags &= ~PBN_BATCH_SPLIT;
    if (flags & ~(PBN_COMPILE_PERT_UNROLLED | PBN_COMPILE_INTERLEAVED | PBN_COMPILE_PIPELINED | PBN_COMPILE_WIDE))
        return fail(PBN_EINVAL, "pbn_batch_compile: unsupported flags 0x%x", flags);
    try {
        std::vector<std::string> functions;
        std::string first_why;
        std::vector<uint32_t> compiled;
        std::vector<uint32_t> tab(b->nets.size(), 0);
        /* networks by descending estimated work: the first kMaxCompiledNets that
         * compile get their own functions */
        std::vector<uint32_t> order(b->nets.size());
        for (uint32_t i = 0; i < (uint32_t)order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
            return b->plans[x]->info.ops_per_step * b->nets[x].n_traj > b->plans[y]->info.ops_per_step * b->nets[y].n_traj;
        });
        for (uint32_t i : order) {
            if (compiled.size() >= kMaxCompiledNets) break;
            const NetDesc& D = b->nets[i];
            pbn::JitBatchNet spec;
            spec.index = i;
            spec.seed = D.seed;
            spec.meta.n_rows = D.n_meta_rows;
            for (uint32_t m = 0; m < D.n_meta_rows; ++m) {
                spec.meta.row[m] = D.meta_row[m];
                spec.meta.mask[m] = D.meta_mask[m];
                spec.meta.val[m] = D.meta_val[m];
            }
            std::string fn, why;
            if (pbn::jit_batch_function(b->plans[i], flags, spec, &fn, &tab[i], &why)) {
                functions.push_back(std::move(fn));
                compiled.push_back(i);
            } else if (first_why.empty()) {
                first_why = why;
            }
        }
        if (compiled.empty())
            return fail(PBN_EINVAL, "pbn_batch_compile: no network of the batch compiles (%s)", first_why.c_str());
        std::sort(compiled.begin(), compiled.end());
        /* split: the module holds only compiled networks; the others run in the
         * library's 1,024-thread kernel, with their items shaped for it */
        const bool interp = !split && compiled.size() < b->nets.size();
        std::vector<NetDesc> wide_desc;
        if (split) {
            std::vector<uint8_t> is_c(b->nets.size(), 0);
            for (uint32_t i : compiled) is_c[i] = 1;
            wide_desc = b->nets;
            for (uint32_t i = 0; i < (uint32_t)b->nets.size(); ++i)
                if (!is_c[i] && interp_shape(b->plans[i], 1024, !b->lane_groups, &wide_desc[i]) != PBN_OK)
                    return fail(PBN_ETOOBIG, "pbn_batch_compile: network %u does not fit a 1,024-thread CTA", i);
        }
        void *lib = nullptr, *kern = nullptr;
        double ms = 0;
        std::string log;
        const int rc = pbn::jit_batch_module(functions, compiled, interp, b->threads, &lib, &kern, &ms, &log);
        if (rc != PBN_OK) return rc;
        if (split) b->nets = wide_desc;
        b->split = split;
        /* compiled networks: one trajectory per thread, their tables (when the code
         * reads them from shared memory) staged from the plan image */
        for (uint32_t i : compiled) {
            NetDesc& D = b->nets[i];
            D.compiled = 1;
            D.lg = 1;
            D.nt = b->threads;
            D.specs_in_smem = 0;
            D.tables_in_smem = tab[i] ? 1u : 0u;
            D.stage_bytes = tab[i];
            D.stage_off = tab[i] ? D.off_tables : 0u;
            D.smem_state_off = 0;
        }
        cut_items(b);
        b->module = lib;
        b->module_kernel = kern;
        {
            /* a new kernel: its occupancy is found again on each device */
            std::lock_guard<std::mutex> g(b->mu);
            for (int d = 0; d < kMaxDevices; ++d) b->occ_per_sm[d] = b->sms[d] = b->occ_i[d] = 0;
        }
        if (compile_ms) *compile_ms = ms;
        return PBN_OK;
    } catch (const std::bad_alloc&) {
        return fail(PBN_ENOMEM, "pbn_batch_compile: out of memory");
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
/* The batch's kernel: its compiled module's dispatcher, or the library's for its
 * CTA size. */
const void* batch_kernel(const pbn_batch* b) {
    if (b->module_kernel) return b->module_kernel;
    return b->threads == 1024 ? pbn::batch_kernel_1024() : reinterpret_cast<const void*>(pbn_batch_kernel);
}

/* One persistent launch of a batch: a kernel, its CTA size and shared memory, and
 * the range of work items it takes. */
struct Part {
    const void* kern;
    uint32_t threads;
    size_t smem;
    uint32_t first, count;
    bool interp_1024;  /* the split batch's interpreter part (its own occupancy record) */
};

/* The launches of a batch: one, or for a split batch the compiled networks' items
 * (module kernel) and then the interpreted ones (1,024-thread kernel). */
std::vector<Part> batch_parts(const pbn_batch* b) {
    std::vector<Part> parts;
    if (!b->split) {
        parts.push_back(Part{batch_kernel(b), b->threads, b->info.smem_bytes, 0u, b->info.n_items, false});
        return parts;
    }
    if (b->n_items_c) parts.push_back(Part{b->module_kernel, 512u, b->smem_c, 0u, b->n_items_c, false});
    if (b->info.n_items > b->n_items_c)
        parts.push_back(Part{pbn::batch_kernel_1024(), 1024u, b->smem_i, b->n_items_c, b->info.n_items - b->n_items_c, true});
    return parts;
}

/* Grid of one part on the current device: raises the kernel's shared-memory limit
 * there to the part's need (never lowering what another batch set), and finds the
 * CTAs per SM and the SM count of that device on the batch's first run on it. */
int launch_shape(const pbn_batch* b, const Part& pt, uint32_t ctas_per_sm, const char* who, uint32_t* grid) {
    using pbn::fail;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(PBN_ECUDA, "%s: %s", who, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(PBN_EINVAL, "%s: device %d beyond %d", who, dev, kMaxDevices);
    const int se = pbn::ensure_dyn_smem(pt.kern, pt.smem);
    if (se != 0) return fail(PBN_ECUDA, "%s: %s", who, cudaGetErrorString(static_cast<cudaError_t>(se)));
    int per_sm = 0, sms = 0;
    {
        std::lock_guard<std::mutex> g(b->mu);
        int* occ = pt.interp_1024 ? &b->occ_i[dev] : &b->occ_per_sm[dev];
        if (!*occ) {
            int o = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, pt.kern, (int)pt.threads, pt.smem);
            if (e != cudaSuccess || o < 1) return fail(PBN_ETOOBIG, "%s: the batch kernel does not fit an SM", who);
            *occ = o;
        }
        if (!b->sms[dev]) b->sms[dev] = pbn::device_sms();
        per_sm = *occ;
        sms = b->sms[dev];
    }
    if (ctas_per_sm && (int)ctas_per_sm < per_sm) per_sm = (int)ctas_per_sm;
    *grid = (uint32_t)std::min<uint64_t>((uint64_t)sms * per_sm, std::max<uint32_t>(1u, pt.count));
    return PBN_OK;
}

/* Every launch of the batch on `st`, one after the other on the same queue (the last
 * CTA of each launch resets it for the next). */
int launch_all(const pbn_batch* b, BatchParams P, uint32_t ctas_per_sm, const char* who, cudaStream_t st) {
    using pbn::fail;
    const WorkItem* items = P.items;
    for (const Part& pt : batch_parts(b)) {
        uint32_t grid = 0;
        const int rc = launch_shape(b, pt, ctas_per_sm, who, &grid);
        if (rc != PBN_OK) return rc;
        P.items = items + pt.first;
        P.n_items = pt.count;
        void* args[] = {&P};
        const cudaError_t e = cudaLaunchKernel(pt.kern, dim3(grid), dim3(pt.threads), args, pt.smem, st);
        if (e != cudaSuccess) return fail(PBN_ECUDA, "%s: %s", who, cudaGetErrorString(e));
    }
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
    return launch_all(b, P, ctas_per_sm, "pbn_batch_run", static_cast<cudaStream_t>(stream));
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
    return launch_all(b, P, ctas_per_sm, "pbn_batch_run_static", st);
}
