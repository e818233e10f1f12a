/*
 * pbn_sim.cu -- sm_103a kernel of the structure-based PBN simulation
 * (Algorithm 5, ParallelSimulation, with the step semantics of Eq. 1).
 *
 * One trajectory is handled by LG lanes of a warp (a lane group).  Per CTA:
 *   - the plan image (group specs, thresholds, maps and, when they fit, the merged
 *     tables) is bulk-copied global -> shared by one thread with cp.async.bulk,
 *     completion tracked by an mbarrier (bounded wait);
 *   - the grouped state of each trajectory lives in shared memory as 32-bit rows
 *     S[buf][row][slot] (double buffered), so that all lanes of a warp reading the
 *     same row touch consecutive banks.
 * Per step t and trajectory (Philox4x32-10 keyed by (seed, trajectory, t)):
 *   1. perturbation (Sec. 3.2, Step 2): every original 64-node word draws its
 *      Bernoulli(P / 2^32) lanes bit-sliced, most significant level first, and
 *      stops once every lane is decided.  Any set lane means a perturbed step
 *      (leaves included, which replaces Algorithm 1's single draw); the set lanes
 *      of retained nodes are flipped in the grouped state.
 *   2. otherwise (Sec. 3.3, Step 3): the SEL blocks of the retained multi-function
 *      nodes are drawn into shared memory; for every group the combined choice c
 *      (mixed radix over its multi-function nodes), the input pattern x and the
 *      table entry T[c][x] give the group's new bits, ORed into the next state at
 *      the group's offset (cum in Algorithm 5).
 *   3. the meta-state indicator z of the new state updates the per-trajectory
 *      counts V, n01, n10, n11 of the two-state chain (Sec. 4.2).
 * Perturbed steps only flip bits; they never evaluate predictor functions (Eq. 1).
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "pbn_device.cuh"
#include "pbn_interp.cuh"
#include "pbn_internal.h"
#include "pbn_team.cuh"

namespace {

constexpr uint32_t kWeyl0 = 0x9E3779B9u;
constexpr uint32_t kWeyl1 = 0xBB67AE85u;
constexpr int kMaxMetaRows = 16;
constexpr uint32_t kMaxCtaThreads = 1024;
constexpr size_t kStaticSmemReserve = 1024;

struct SimParams {
    const uint8_t* image;      /* device copy of the plan image */
    uint64_t* state;           /* [W64][n_traj] */
    uint64_t* counts;          /* [5][n_traj] or null */
    unsigned long long* pooled;/* [5] or null */
    uint32_t* status;          /* or null */
    uint64_t* trace;           /* [n_steps][W64][n_traj] or null */
    uint64_t traj_begin;
    uint64_t step_begin;
    uint32_t key0[10];         /* Philox key schedule, round r: seed + r * Weyl */
    uint32_t key1[10];
    uint32_t n_traj;
    uint32_t n_steps;
    uint32_t kv0;              /* first step whose resulting state is counted */
    uint32_t kp0;              /* first step whose (before, after) pair is counted */
    uint32_t pairs;            /* counted pairs of this launch (n00 = pairs - others) */
    uint32_t count_first;      /* 1: the keyed s(0) itself is counted (count_from = 0) */
    uint32_t init;             /* 0: keyed s(0), 1: read state */
    uint32_t nt;               /* trajectory slots per CTA */
    uint32_t stage_bytes;      /* image bytes staged into shared memory */
    uint32_t image_bytes;      /* total image bytes (checked against the header) */
    uint32_t smem_state_off;   /* byte offset of the state rows in dynamic smem */
    uint32_t hmax;             /* level pairs that can still decide a perturbation */
    uint32_t n, W, W32, n_sel, P;
    uint32_t off_words, off_groups, off_multi, off_selslot, off_thr, off_inputs, off_selblk, off_gorder, off_ret, off_pos,
        off_tables, n_groups, off_subs, per_node, sampler, off_geo, off_wgroups;
    uint64_t geo_full, geo_last;  /* geometric sampler: thresholds of a full and the last word */
    uint32_t n_meta_rows;
    uint32_t trace_stride;     /* steps between trace snapshots (>= 1) */
    uint32_t team_warps;       /* team kernel: warps per team */
    uint32_t team_tpl;         /* team kernel: trajectories per lane (a team of 32 x this many) */
    uint32_t meta_row[kMaxMetaRows];
    uint32_t meta_mask[kMaxMetaRows];
    uint32_t meta_val[kMaxMetaRows];
};

/* up to 1024 threads per CTA (64 registers a thread): a plan whose specs fill most of
 * shared memory runs one CTA per SM, and its warps are then all the SM has */
template <int LG, bool TRACE, bool TAB_SMEM>
__global__ void __launch_bounds__(kMaxCtaThreads) pbn_sim_kernel(const SimParams P) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t stage_bar;

    /* ---- stage the plan image into shared memory (bulk copy, bounded wait) ---- */
    if (!pbn_stage(smem, P.image, P.stage_bytes, &stage_bar)) {
        if (threadIdx.x == 0 && P.status) atomicOr(P.status, PBN_DEV_STAGE_TIMEOUT);
        return;
    }
    const pbn_img_header* hdr = reinterpret_cast<const pbn_img_header*>(smem);
    if (hdr->magic != PBN_IMG_MAGIC || hdr->image_bytes != P.image_bytes || hdr->n != P.n ||
        hdr->W32 != P.W32 || hdr->n_sel != P.n_sel || hdr->off_tables != P.off_tables) {
        if (threadIdx.x == 0 && P.status) atomicOr(P.status, PBN_DEV_BAD_PLAN);
        return;
    }
    const uint32_t slot = threadIdx.x / LG;
    const uint32_t lane = LG == 1 ? 0u : (threadIdx.x % LG);
    const uint64_t lt = (uint64_t)blockIdx.x * P.nt + slot;
    const bool active = lt < P.n_traj;
    uint32_t c[4] = {0, 0, 0, 0};
    pbn_interp_run<LG, TRACE, TAB_SMEM, true>(P, smem, P.smem_state_off, P.nt, slot, lane, lt, active, c);
    const uint32_t cV = c[0], c01 = c[1], c10 = c[2], c11 = c[3];

    /* ---- pooled counts: warp reduction, one atomic per warp and count ---- */
    if (P.pooled) {
        const bool lead = active && lane == 0;
        uint64_t v[5] = {lead ? cV : 0u, lead ? (uint64_t)(P.pairs - c01 - c10 - c11) : 0u,
                         lead ? c01 : 0u, lead ? c10 : 0u, lead ? c11 : 0u};
#pragma unroll
        for (int i = 0; i < 5; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xFFFFFFFFu, v[i], o);
        }
        if ((threadIdx.x & 31u) == 0) {
#pragma unroll
            for (int i = 0; i < 5; ++i)
                if (v[i]) atomicAdd(P.pooled + i, (unsigned long long)v[i]);
        }
    }
}

template <int LG, bool TRACE, bool TAB_SMEM>
cudaError_t launch_t(const SimParams& P, uint32_t grid, uint32_t tpb, size_t smem, cudaStream_t st) {
    auto kern = pbn_sim_kernel<LG, TRACE, TAB_SMEM>;
    const int e = pbn::ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != 0) return static_cast<cudaError_t>(e);
    kern<<<grid, tpb, smem, st>>>(P);
    return cudaGetLastError();
}

/* The team interpreter (pbn_team.cuh): a CTA of P.nt / (32 TPL) teams of
 * P.team_warps warps, 32 TPL trajectories a team, the staged records at the start of
 * shared memory and the teams' states after them. */
template <int TPL, bool TRACE, bool TAB_SMEM>
__global__ void __launch_bounds__(kMaxCtaThreads) pbn_team_kernel(const SimParams P) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t stage_bar;
    if (!pbn_stage(smem, P.image, P.stage_bytes, &stage_bar)) {
        if (threadIdx.x == 0 && P.status) atomicOr(P.status, PBN_DEV_STAGE_TIMEOUT);
        return;
    }
    const pbn_img_header* hdr = reinterpret_cast<const pbn_img_header*>(smem);
    if (hdr->magic != PBN_IMG_MAGIC || hdr->image_bytes != P.image_bytes || hdr->n != P.n ||
        hdr->W32 != P.W32 || hdr->n_sel != P.n_sel || hdr->off_tables != P.off_tables) {
        if (threadIdx.x == 0 && P.status) atomicOr(P.status, PBN_DEV_BAD_PLAN);
        return;
    }
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t K = P.team_warps;
    const uint32_t team = warp / K, wt = warp - team * K;
    const uint64_t lt0 = (uint64_t)blockIdx.x * P.nt + team * 32u * TPL + lane;
    uint32_t act = 0;
#pragma unroll
    for (int j = 0; j < TPL; ++j) act |= (lt0 + 32u * j < P.n_traj ? 1u : 0u) << j;
    uint8_t* const tsm = smem + P.smem_state_off + team * pbn_team_smem_bytes(P.W32, P.n_sel, TPL);
    uint32_t c[4 * TPL];
    pbn_team_run<TPL, TRACE, TAB_SMEM>(P, smem, tsm, K, wt, lane, lt0, act, c);
    if (P.pooled) {
        uint64_t v[5] = {0, 0, 0, 0, 0};
        if (wt == 0) {
#pragma unroll
            for (int j = 0; j < TPL; ++j) {
                if (!((act >> j) & 1u)) continue;
                v[0] += c[4 * j];
                v[1] += P.pairs - c[4 * j + 1] - c[4 * j + 2] - c[4 * j + 3];
                v[2] += c[4 * j + 1];
                v[3] += c[4 * j + 2];
                v[4] += c[4 * j + 3];
            }
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xFFFFFFFFu, v[i], o);
        }
        if (lane == 0 && wt == 0) {
#pragma unroll
            for (int i = 0; i < 5; ++i)
                if (v[i]) atomicAdd(P.pooled + i, (unsigned long long)v[i]);
        }
    }
}

template <int TPL, bool TRACE, bool TAB_SMEM>
cudaError_t launch_team_t(const SimParams& P, uint32_t grid, uint32_t tpb, size_t smem, cudaStream_t st) {
    auto kern = pbn_team_kernel<TPL, TRACE, TAB_SMEM>;
    const int e = pbn::ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    if (e != 0) return static_cast<cudaError_t>(e);
    kern<<<grid, tpb, smem, st>>>(P);
    return cudaGetLastError();
}

template <int TPL>
cudaError_t launch_team_tpl(const SimParams& P, bool trace, bool tab_smem, uint32_t grid, uint32_t tpb, size_t smem,
                            cudaStream_t st) {
    if (trace) return tab_smem ? launch_team_t<TPL, true, true>(P, grid, tpb, smem, st)
                               : launch_team_t<TPL, true, false>(P, grid, tpb, smem, st);
    return tab_smem ? launch_team_t<TPL, false, true>(P, grid, tpb, smem, st)
                    : launch_team_t<TPL, false, false>(P, grid, tpb, smem, st);
}

template <int LG>
cudaError_t launch_lg(const SimParams& P, bool trace, bool tab_smem, uint32_t grid, uint32_t tpb, size_t smem,
                      cudaStream_t st) {
    if (trace) return tab_smem ? launch_t<LG, true, true>(P, grid, tpb, smem, st)
                               : launch_t<LG, true, false>(P, grid, tpb, smem, st);
    return tab_smem ? launch_t<LG, false, true>(P, grid, tpb, smem, st)
                    : launch_t<LG, false, false>(P, grid, tpb, smem, st);
}

}  // namespace

/* ---- per-device launch facts and shared-memory opt-in ------------------------------ */
namespace pbn {
namespace {
constexpr int kMaxDevices = 64;
struct DeviceFacts {
    int sms = 0, smem_optin = 0;
};
std::mutex g_dev_mu;
DeviceFacts g_dev[kMaxDevices];
std::map<std::pair<int, const void*>, size_t> g_smem_set; /* (device, kernel) -> limit set */

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    return dev;
}

const DeviceFacts& facts() {
    const int dev = current_device();
    std::lock_guard<std::mutex> g(g_dev_mu);
    DeviceFacts& F = g_dev[dev];
    if (!F.sms) {
        int v = 0;
        F.sms = (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0) ? v : 1;
        F.smem_optin = (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess && v > 0)
                           ? v
                           : 48 * 1024;
    }
    return F;
}
}  // namespace

int device_sms() { return facts().sms; }
int device_smem_optin() { return facts().smem_optin; }

int ensure_dyn_smem(const void* func, size_t bytes, size_t static_bytes) {
    if (bytes + static_bytes <= 48u * 1024u) return 0;
    const int dev = current_device();
    std::lock_guard<std::mutex> g(g_dev_mu);
    size_t& set = g_smem_set[std::make_pair(dev, func)];
    if (bytes <= set) return 0;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError(); /* reported here: not left for the next launch's check */
        return (int)e;
    }
    set = bytes;
    return 0;
}
}  // namespace pbn

namespace {
int device_smem_limit() { return pbn::device_smem_optin(); }
int device_sm_count() { return pbn::device_sms(); }
}  // namespace

namespace pbn {
int jit_launch(const pbn_plan* plan, pbn_jit_params* P, uint32_t n_traj, int sms, cudaStream_t st);
}

extern "C" int pbn_simulate(const pbn_plan* plan, const void* d_image, const pbn_sim_args* a, void* stream) {
    using pbn::fail;
    if (!plan || !a) return fail(PBN_EINVAL, "pbn_simulate: NULL argument");
    if (a->n_traj == 0) return PBN_OK;
    if (!d_image || ((uintptr_t)d_image & 15u)) return fail(PBN_EINVAL, "pbn_simulate: d_image must be 16-byte aligned device memory");
    if (!a->d_state) return fail(PBN_EINVAL, "pbn_simulate: d_state is required");
    if (a->n_traj >= (1ull << 31)) return fail(PBN_EINVAL, "pbn_simulate: n_traj must be < 2^31");
    if (a->n_steps >= (1ull << 32)) return fail(PBN_EINVAL, "pbn_simulate: n_steps must be < 2^32");
    if (a->traj_begin + a->n_traj > (1ull << 48)) return fail(PBN_EINVAL, "pbn_simulate: trajectory ids must be < 2^48");
    if (a->step_begin + a->n_steps > (1ull << 48)) return fail(PBN_EINVAL, "pbn_simulate: step indices must be < 2^48");
    if (a->init != PBN_INIT_KEYED && a->init != PBN_INIT_STATE) return fail(PBN_EINVAL, "pbn_simulate: bad init mode");
    if (a->init == PBN_INIT_KEYED && a->step_begin != 0) return fail(PBN_EINVAL, "pbn_simulate: keyed initial state needs step_begin == 0");
    if (a->kernel > PBN_KERNEL_TEAM) return fail(PBN_EINVAL, "pbn_simulate: unknown kernel selector %u", a->kernel);
    if (a->n_meta < 1 || a->n_meta > 1024 || !a->meta_ids) return fail(PBN_EINVAL, "pbn_simulate: need 1..1024 meta-state nodes");
    const uint32_t tstride = a->trace_stride ? a->trace_stride : 1u;
    if (a->d_trace && (a->n_steps / tstride) * (uint64_t)plan->info.state_words * a->n_traj >= (1ull << 40))
        return fail(PBN_EINVAL, "pbn_simulate: trace too large");

    const pbn_img_header& H = plan->hdr;
    SimParams P;
    memset(&P, 0, sizeof(P));
    /* meta-state: mask and value per state row */
    {
        pbn::MetaRows M;
        const int rc = pbn::meta_rows(plan, a->meta_ids, a->meta_vals, a->n_meta, kMaxMetaRows, "pbn_simulate", &M);
        if (rc != PBN_OK) return rc;
        P.n_meta_rows = M.n_rows;
        for (uint32_t k = 0; k < M.n_rows; ++k) {
            P.meta_row[k] = M.row[k];
            P.meta_mask[k] = M.mask[k];
            P.meta_val[k] = M.val[k];
        }
    }

    P.image = static_cast<const uint8_t*>(d_image);
    P.state = static_cast<uint64_t*>(a->d_state);
    P.counts = static_cast<uint64_t*>(a->d_counts);
    P.pooled = static_cast<unsigned long long*>(a->d_pooled);
    P.status = static_cast<uint32_t*>(a->d_status);
    P.trace = static_cast<uint64_t*>(a->d_trace);
    P.trace_stride = tstride;
    P.traj_begin = a->traj_begin;
    P.step_begin = a->step_begin;
    const uint32_t k0 = (uint32_t)a->seed, k1 = (uint32_t)(a->seed >> 32);
    for (int r = 0; r < 10; ++r) {
        P.key0[r] = k0 + (uint32_t)r * kWeyl0;
        P.key1[r] = k1 + (uint32_t)r * kWeyl1;
    }
    P.n_traj = (uint32_t)a->n_traj;
    P.n_steps = (uint32_t)a->n_steps;
    /* counting window: the states this launch produces, s(u) for u in
     * (step_begin, step_begin + n_steps], are counted iff u >= count_from, the pairs
     * (s(t), s(t+1)) it steps through iff t >= count_from, and its initial state only
     * when the launch starts the trajectory (keyed s(0), count_from = 0); a resumed
     * launch never recounts the state the launch before it produced, so the counts
     * of a chain of launches are those of one launch over all its steps */
    const uint64_t sb = a->step_begin, cf = a->count_from, ns = a->n_steps;
    const uint64_t kv0 = cf > sb + 1 ? cf - sb - 1 : 0;
    const uint64_t kp0 = cf > sb ? cf - sb : 0;
    P.kv0 = (uint32_t)(kv0 < ns ? kv0 : ns);
    P.kp0 = (uint32_t)(kp0 < ns ? kp0 : ns);
    P.pairs = (uint32_t)(ns - P.kp0);
    P.count_first = (a->init == PBN_INIT_KEYED && cf == 0) ? 1u : 0u;
    P.init = a->init;
    P.n = H.n;
    P.W = H.W;
    P.W32 = H.W32;
    P.n_sel = H.n_sel;
    P.P = H.P;
    P.off_words = H.off_words;
    P.off_groups = H.off_groups;
    P.off_multi = H.off_multi;
    P.off_selslot = H.off_selslot;
    P.off_gorder = H.off_gorder;
    P.off_wgroups = H.off_wgroups;
    P.off_subs = H.off_subs;
    P.per_node = H.semantics == PBN_SEM_NODEWISE ? 1u : 0u;
    P.sampler = H.sampler;
    P.off_geo = H.off_geo;
    {
        const uint64_t* G = reinterpret_cast<const uint64_t*>(plan->image.data() + H.off_geo);
        const uint32_t nl = H.n & 63u;
        P.geo_full = G[63];
        P.geo_last = G[(nl ? nl : 64u) - 1];
    }
    P.n_groups = H.n_groups;
    P.off_thr = H.off_thr;
    P.off_inputs = H.off_inputs;
    P.off_selblk = H.off_selblk;
    P.off_ret = H.off_ret;
    P.off_pos = H.off_pos;
    P.off_tables = H.off_tables;
    P.stage_bytes = H.stage_bytes;
    P.image_bytes = H.image_bytes;
    P.smem_state_off = (H.stage_bytes + 127u) & ~127u;
    /* levels after the last set bit of P only retire lanes: the outcome is fixed */
    P.hmax = H.P ? (31u - (uint32_t)__builtin_ctz(H.P)) / 2u + 1u : 0u;

    const int sms = device_sm_count();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (a->kernel == PBN_KERNEL_COMPILED) {
        const int rc = pbn::jit_compile(plan, pbn::jit_current_flags(plan));
        if (rc) return rc;
    }
    if (a->kernel == PBN_KERNEL_COMPILED ||
        (a->kernel == PBN_KERNEL_AUTO && a->lanes_per_traj <= 1 && a->trajs_per_block == 0 && pbn::jit_ready(plan))) {
        pbn_jit_params J;
        memset(&J, 0, sizeof(J));
        J.image = P.image;
        J.state = P.state;
        J.counts = P.counts;
        J.pooled = P.pooled;
        J.status = P.status;
        J.trace = P.trace;
        J.trace_stride = P.trace_stride;
        J.traj_begin = P.traj_begin;
        J.step_begin = P.step_begin;
        memcpy(J.key0, P.key0, sizeof(J.key0));
        memcpy(J.key1, P.key1, sizeof(J.key1));
        J.n_traj = P.n_traj;
        J.n_steps = P.n_steps;
        J.kv0 = P.kv0;
        J.kp0 = P.kp0;
        J.pairs = P.pairs;
        J.count_first = P.count_first;
        J.init = P.init;
        J.off_tables = P.off_tables;
        J.off_ret = P.off_ret;
        J.off_pos = P.off_pos;
        J.image_bytes = P.image_bytes;
        for (uint32_t m = 0; m < P.n_meta_rows; ++m) {
            J.meta_mask[P.meta_row[m]] = P.meta_mask[m];
            J.meta_val[P.meta_row[m]] = P.meta_val[m];
        }
        return pbn::jit_launch(plan, &J, P.n_traj, sms, st);
    }

    /* dynamic shared memory a CTA may take: the opt-in limit less a reserve for the
     * kernels' static shared memory (a stage barrier and a few words) */
    const size_t smem_lim = (size_t)device_smem_limit() - kStaticSmemReserve;
    if (a->kernel == PBN_KERNEL_TEAM) {
        /* teams of K warps on 32 TPL trajectories (TPL per lane: 2 when such a team
         * fits, so that each record decode serves two trajectories): T teams per CTA
         * (T x K <= 32 warps), by default as many as the shared memory holds up to one
         * wave of CTAs over the SMs, and K = 32 / T */
        if (P.per_node) return fail(PBN_EINVAL, "pbn_simulate: the team kernel runs Eq. 1 semantics only");
        if (a->team_warps > 32u || a->team_trajs_per_lane > 2u)
            return fail(PBN_EINVAL, "pbn_simulate: team kernel needs <= 32 warps and 1 or 2 trajectories per lane");
        const size_t fixed = P.smem_state_off;
        uint32_t tpl = a->team_trajs_per_lane;
        if (tpl == 0) tpl = fixed + pbn_team_smem_bytes(H.W32, H.n_sel, 2) <= smem_lim ? 2u : 1u;
        const uint32_t per_team = 32u * tpl;
        if (a->trajs_per_block % per_team || a->trajs_per_block > 32u * per_team)
            return fail(PBN_EINVAL, "pbn_simulate: team kernel needs trajs_per_block a multiple of %u", per_team);
        const size_t tb = pbn_team_smem_bytes(H.W32, H.n_sel, tpl);
        if (fixed + tb > smem_lim)
            return fail(PBN_ETOOBIG, "pbn_simulate: a team needs %zu bytes of shared memory", fixed + tb);
        const uint32_t tmax = (uint32_t)std::min<size_t>(32, (smem_lim - fixed) / tb);
        const uint64_t n_teams = (a->n_traj + per_team - 1) / per_team;
        uint32_t T = a->trajs_per_block / per_team;
        if (T == 0)
            T = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(tmax, (n_teams + sms - 1) / (uint64_t)sms));
        uint32_t K = a->team_warps ? a->team_warps : std::max(1u, 32u / T);
        if (T > tmax) return fail(PBN_ETOOBIG, "pbn_simulate: %u teams exceed the shared memory of a CTA", T);
        if (T * K > 32u) return fail(PBN_EINVAL, "pbn_simulate: %u teams of %u warps exceed 1,024 threads", T, K);
        P.team_warps = K;
        P.team_tpl = tpl;
        P.nt = per_team * T;
        const uint64_t grid = (a->n_traj + P.nt - 1) / P.nt;
        const size_t smem = fixed + (size_t)T * tb;
        const bool tr = a->d_trace != nullptr, ts = H.tables_in_smem != 0;
        const cudaError_t e = tpl == 2 ? launch_team_tpl<2>(P, tr, ts, (uint32_t)grid, 32u * K * T, smem, st)
                                       : launch_team_tpl<1>(P, tr, ts, (uint32_t)grid, 32u * K * T, smem, st);
        if (e != cudaSuccess) return fail(PBN_ECUDA, "pbn_simulate: %s", cudaGetErrorString(e));
        return PBN_OK;
    }

    /* launch shape: lanes per trajectory and trajectory slots per CTA */
    uint32_t LG = a->lanes_per_traj;
    const size_t per_traj = plan->per_traj_smem;
    const size_t fixed = P.smem_state_off;
    if (LG == 0) {
        /* one lane per trajectory when the SMs fill with trajectories; otherwise
         * lane groups (they split the perturbation words, SEL blocks and groups of
         * a trajectory) until a CTA holds 8 to 16 warps.  States of 32 words or more
         * keep doubling up to a warp per trajectory while the trajectories that fit
         * would fill a CTA of 1,024 threads (on a 62-word state 32 lanes ran 1.26x
         * faster than 16 and 1.66x faster than 8) */
        LG = 1;
        const uint64_t per_sm = (a->n_traj + sms - 1) / sms;
        const uint64_t fit = fixed + per_traj * 32 <= smem_lim ? (smem_lim - fixed) / per_traj : 32;
        const uint64_t slots = std::min<uint64_t>(per_sm, std::min<uint64_t>(fit, 512));
        while (LG < 8 && slots * LG < 256 && H.W32 >= 4 * LG) LG *= 2;
        if (H.W32 >= 32) {
            while (LG < 32 && 2 * LG <= H.W32 && slots * LG < kMaxCtaThreads) LG *= 2;
        } else if (LG > 1 && slots * LG < 512 && LG < 8 && H.W32 >= 4 * LG) {
            LG *= 2;
        }
    }
    if (LG == 0 || LG > 32 || (LG & (LG - 1)))
        return fail(PBN_EINVAL, "pbn_simulate: lanes_per_traj must be 1, 2, 4, 8, 16 or 32");
    if (fixed + per_traj * (32 / LG) > smem_lim)
        return fail(PBN_ETOOBIG, "pbn_simulate: plan needs %zu bytes of shared memory for one warp", fixed + per_traj * (32 / LG));
    uint32_t nt = a->trajs_per_block;
    if (nt == 0) {
        /* k CTAs per SM, trajectories spread evenly: the grid is close to a multiple
         * of the SM count, with at most kMaxCtaThreads threads per CTA */
        const uint32_t unit = 32 / LG; /* trajectories per warp */
        for (uint64_t k = 1;; ++k) {
            uint64_t want = (a->n_traj + (uint64_t)sms * k - 1) / ((uint64_t)sms * k);
            want = ((want + unit - 1) / unit) * unit;
            if (want * LG <= kMaxCtaThreads && fixed + per_traj * want <= smem_lim) {
                nt = (uint32_t)want;
                break;
            }
            if (want <= unit) {
                nt = unit;
                break;
            }
        }
    }
    if ((nt * LG) % 32 != 0 || nt * LG > kMaxCtaThreads || nt == 0)
        return fail(PBN_EINVAL, "pbn_simulate: trajs_per_block * lanes_per_traj must be a multiple of 32 and <= 1024");
    const size_t smem = fixed + per_traj * nt;
    if (smem > smem_lim) return fail(PBN_ETOOBIG, "pbn_simulate: %zu bytes of shared memory exceed the device limit", smem);
    P.nt = nt;
    const uint64_t grid = (a->n_traj + nt - 1) / nt;
    cudaError_t e;
    const bool tr = a->d_trace != nullptr;
    const bool ts = H.tables_in_smem != 0;
    switch (LG) {
        case 1: e = launch_lg<1>(P, tr, ts, (uint32_t)grid, nt * LG, smem, st); break;
        case 2: e = launch_lg<2>(P, tr, ts, (uint32_t)grid, nt * LG, smem, st); break;
        case 4: e = launch_lg<4>(P, tr, ts, (uint32_t)grid, nt * LG, smem, st); break;
        case 8: e = launch_lg<8>(P, tr, ts, (uint32_t)grid, nt * LG, smem, st); break;
        case 16: e = launch_lg<16>(P, tr, ts, (uint32_t)grid, nt * LG, smem, st); break;
        default: e = launch_lg<32>(P, tr, ts, (uint32_t)grid, nt * LG, smem, st); break;
    }
    if (e != cudaSuccess) return fail(PBN_ECUDA, "pbn_simulate: %s", cudaGetErrorString(e));
    return PBN_OK;
}
