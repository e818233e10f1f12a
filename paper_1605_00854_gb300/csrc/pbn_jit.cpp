/*
 * pbn_jit.cpp -- compiled plans: a plan's Preparation output (Algorithm 5: the
 * groups, their merged tables, the selection thresholds and the perturbation
 * threshold) is turned into the source of a kernel in which all of it is constant,
 * compiled for sm_103a with NVRTC and launched with the runtime's library API.
 *
 * Compared with the interpreter kernel (pbn_sim.cu), the state lives in registers,
 * input gathers are constant shifts and masks, the selection thresholds and the
 * levels of P are immediates, and merged tables of at most 64 bits are immediates
 * too; larger tables are staged into shared memory by a bulk copy.  The step
 * semantics (Eq. 1, or the plan's node-wise variant) and the keyed draws (of the
 * plan's perturbation sampler) are identical, so the results are bit for bit those
 * of the interpreter and of the unreduced definition.  Flags choose the code shape:
 * how the perturbation levels are scheduled, multiply gathers, and the wide form
 * for plans with many SEL blocks.
 *
 * Compilation costs host time (tens to hundreds of milliseconds), which pays off
 * for long runs of one network, as the paper observes for its own pre-processing
 * (Sec. 4.1, Table 1).
 */
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <vector>

#include "pbn_device.cuh"
#include "pbn_internal.h"

namespace {

const char kDeviceHeader[] =
#include "pbn_device_cuh.inc"
    ;

/* ---- NVRTC, loaded on first use --------------------------------------------------- */
typedef int nvrtcResult_t;
typedef struct _nvrtcProgram* nvrtcProgram_t;
struct Nvrtc {
    nvrtcResult_t (*create)(nvrtcProgram_t*, const char*, const char*, int, const char* const*, const char* const*);
    nvrtcResult_t (*compile)(nvrtcProgram_t, int, const char* const*);
    nvrtcResult_t (*log_size)(nvrtcProgram_t, size_t*);
    nvrtcResult_t (*log)(nvrtcProgram_t, char*);
    nvrtcResult_t (*cubin_size)(nvrtcProgram_t, size_t*);
    nvrtcResult_t (*cubin)(nvrtcProgram_t, char*);
    nvrtcResult_t (*destroy)(nvrtcProgram_t*);
    bool ok = false;
    std::string err;
};

Nvrtc& nvrtc() {
    static Nvrtc N;
    static std::once_flag once;
    std::call_once(once, [] {
        const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                               "/usr/local/cuda/lib64/libnvrtc.so"};
        void* h = nullptr;
        for (const char* nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) {
            N.err = "libnvrtc not found";
            return;
        }
#define PBN_SYM(field, name)                                          \
    *reinterpret_cast<void**>(&N.field) = dlsym(h, name);             \
    if (!N.field) {                                                   \
        N.err = std::string("libnvrtc lacks ") + name;                \
        return;                                                       \
    }
        PBN_SYM(create, "nvrtcCreateProgram");
        PBN_SYM(compile, "nvrtcCompileProgram");
        PBN_SYM(log_size, "nvrtcGetProgramLogSize");
        PBN_SYM(log, "nvrtcGetProgramLog");
        PBN_SYM(cubin_size, "nvrtcGetCUBINSize");
        PBN_SYM(cubin, "nvrtcGetCUBIN");
        PBN_SYM(destroy, "nvrtcDestroyProgram");
#undef PBN_SYM
        N.ok = true;
    });
    return N;
}

/* ---- plan decoding ------------------------------------------------------------------- */
struct View {
    const pbn_img_header* H;
    const uint8_t* img;
    template <class T>
    const T* at(uint32_t off) const { return reinterpret_cast<const T*>(img + off); }
};

std::string hex32(uint32_t v) {
    char b[16];
    snprintf(b, sizeof b, "0x%08xu", v);
    return b;
}

std::string fmt(const char* f, ...) {
    char b[512];
    va_list ap;
    va_start(ap, f);
    vsnprintf(b, sizeof b, f, ap);
    va_end(ap);
    return b;
}

/* Expression selecting bit `bit` of state word s<row> into position b. */
std::string gather(uint32_t row, uint32_t bit, uint32_t b) {
    if (bit == b) return fmt("(s%u & %s)", row, hex32(1u << b).c_str());
    if (bit > b) return fmt("((s%u >> %u) & %s)", row, bit - b, hex32(1u << b).c_str());
    return fmt("((s%u << %u) & %s)", row, b - bit, hex32(1u << b).c_str());
}

const char* lanes = "xyzw";

/* Multiply gather: the k input bits a_0 < ... < a_{k-1} of one state word are moved
 * into a field of `width` bits by one multiplication, field = (((s & mask) * mul) >>
 * shift) & (2^width - 1).  mul is a sum of powers of two that sends bit a_i to a
 * target position t_i >= a_i inside [shift, shift + width); the other partial
 * products and their carries may land anywhere, so a candidate is kept only if the
 * field takes 2^k distinct values over the 2^k input patterns (an injective index:
 * the group's table is rebuilt in that index order).  Candidates are tried in a
 * fixed order (targets in input order, then permutations from a fixed-seed
 * generator), so the generated kernel is deterministic. */
struct MagicTerm {
    uint32_t row, mask, mul, shift, width;
};

uint32_t magic_field(const MagicTerm& t, uint32_t s) {
    return (((s & t.mask) * t.mul) >> t.shift) & ((1u << t.width) - 1u);
}

bool find_magic(uint32_t row, const std::vector<uint32_t>& a, MagicTerm* out) {
    const uint32_t k = (uint32_t)a.size();
    if (k < 3 || k > 8) return false;
    uint32_t mask = 0;
    for (uint32_t x : a) mask |= 1u << x;
    uint64_t rng = 0x9E3779B97F4A7C15ull ^ ((uint64_t)mask << 8) ^ k;
    auto next = [&]() {
        rng ^= rng << 13;
        rng ^= rng >> 7;
        rng ^= rng << 17;
        return rng;
    };
    std::vector<uint8_t> seen;
    for (uint32_t width = k; width <= k; ++width) { /* a perfect field keeps the table size */
        for (uint32_t shift = 0; shift + width <= 32; ++shift) {
            for (int attempt = 0; attempt < 24; ++attempt) {
                /* targets: the first attempt keeps the input order, later ones draw
                 * a random injective placement of the k bits in the field */
                std::vector<uint32_t> slot(width);
                for (uint32_t i = 0; i < width; ++i) slot[i] = i;
                if (attempt)
                    for (uint32_t i = width - 1; i > 0; --i) std::swap(slot[i], slot[next() % (i + 1)]);
                uint32_t mul = 0;
                bool ok = true;
                for (uint32_t i = 0; i < k && ok; ++i) {
                    const uint32_t t = shift + slot[i];
                    if (t < a[i]) ok = false;
                    else mul |= 1u << (t - a[i]); /* equal shifts share one term */
                }
                if (!ok) continue;
                MagicTerm m{row, mask, mul, shift, width};
                seen.assign((size_t)1 << width, 0);
                for (uint32_t x = 0; x < (1u << k) && ok; ++x) {
                    uint32_t sw = 0;
                    for (uint32_t i = 0; i < k; ++i) sw |= ((x >> i) & 1u) << a[i];
                    const uint32_t f = magic_field(m, sw);
                    if (seen[f]) ok = false;
                    seen[f] = 1;
                }
                if (ok) {
                    *out = m;
                    return true;
                }
            }
        }
    }
    return false;
}

struct Generated {
    std::string src;
    uint32_t tab_bytes = 0;  /* bytes of tables staged into shared memory */
    uint32_t warps = 0;      /* warp-split form: warps per CTA (32 trajectories); 0: one trajectory per thread */
    uint32_t dyn_smem = 0;   /* dynamic shared memory to launch with (0: tab_bytes) */
    uint32_t static_smem = 1024; /* upper bound of the kernel's static shared memory */
};

using BatchSpec = pbn::JitBatchNet;

/* The CUDA source of one plan's kernel.  The plan image is read on the host: every
 * gather, threshold, perturbation level and small table becomes an immediate, and
 * the step loop is emitted in the code shape the flags select.  With a BatchSpec the
 * same step loop becomes a device function of a batch module (one work item of the
 * network: one trajectory per thread), with the Philox keys and the meta-state as
 * constants too. */
class KernelSource {
public:
    KernelSource(const pbn_plan& plan, uint32_t flags, const BatchSpec* bs = nullptr)
        : H(plan.hdr), V{&plan.hdr, plan.image.data()}, flags_(bs ? (flags & ~(uint32_t)PBN_COMPILE_MAGIC_GATHER) : flags),
          wide((flags & PBN_COMPILE_WIDE) != 0), bs_(bs), sfx_(bs ? "_" + std::to_string(bs->index) : std::string()) {}

    bool generate(Generated* out, std::string* why) {
        if (flags_ & PBN_COMPILE_WARP_SPLIT) return generate_warp_split(out, why);
        if (!fits(why)) return false;
        bind_sections();
        collect_table_starts();
        plan_multiply_gathers();
        tab_smem = table_bytes <= 48u * 1024u;
        out->tab_bytes = tab_smem ? table_bytes : 0u;
        emit_globals();
        emit_prologue();
        /* the geometric sampler has no level loop to pipeline: its pipelined form is
         * the interleaved one */
        geometric = H.sampler == PBN_PERT_GEOMETRIC;
        pipelined = (flags_ & PBN_COMPILE_PIPELINED) != 0 && !geometric && !wide;
        interleave = !wide && ((flags_ & PBN_COMPILE_INTERLEAVED) != 0 ||
                               ((flags_ & PBN_COMPILE_PIPELINED) != 0 && geometric));
        /* node-wise semantics: every step evaluates the functions and the perturbed
         * nodes (collected in masks) take NOT s */
        nodewise = H.semantics == PBN_SEM_NODEWISE;
        Pv = H.P;
        hmax = Pv ? (31u - (uint32_t)__builtin_ctz(Pv)) / 2u + 1u : 0u;
        if (pipelined) emit_pipelined_steps();
        else emit_steps();
        emit_epilogue();
        out->src = o.str();
        return true;
    }

    /* Warp-split form (PBN_COMPILE_WARP_SPLIT), for wide plans: a CTA of K warps runs
     * 32 trajectories, one per lane, with their grouped states double-buffered in
     * shared memory as S[row][lane] (a warp's accesses to one row are conflict free).
     * Each warp runs straight-line code for its own share of the work: some word pairs
     * of the perturbation draws (phase A: flips XORed into the current state, a
     * per-trajectory "perturbed" flag) and some pairs of state rows (phase B: the SEL
     * blocks and merged groups of those rows, written to the next state; a perturbed
     * trajectory copies its flipped state).  Two CTA barriers per step.  The meta-state
     * indicator is ANDed from each warp's rows into a per-trajectory word and counted
     * by warp 0 one step later.  Draws and results are those of every other form. */
    bool generate_warp_split(Generated* out, std::string* why) {
        if (H.semantics == PBN_SEM_NODEWISE) {
            *why = "the warp-split form takes Eq. 1 semantics only";
            return false;
        }
        if (H.W32 > 128 || H.W > 64) {
            *why = "more than 128 state rows or 4096 original nodes";
            return false;
        }
        bind_sections();
        collect_table_starts();
        gp.assign(H.n_groups, GPlan{}); /* no multiply gathers in this form */
        magic = false;
        tab_smem = table_bytes <= 48u * 1024u;
        out->tab_bytes = tab_smem ? table_bytes : 0u;
        geometric = H.sampler == PBN_PERT_GEOMETRIC;
        interleave = true;
        /* PBN_COMPILE_WS_SELSMEM: the SEL blocks are drawn in phase A, split over the
         * warps by one short loop (thresholds in constant memory), and their choices
         * kept as bytes in shared memory for phase B; otherwise each warp draws the
         * blocks its groups need in its own straight-line code */
        ch_smem_ = (flags_ & PBN_COMPILE_WS_SELSMEM) != 0 && H.n_sel > 0;
        ws_choices_ = !ch_smem_;
        const uint32_t ch_off = ch_smem_ ? ((tab_smem ? table_bytes : 0u) + 127u) & ~127u : 0u;
        const uint32_t ch_bytes = ch_smem_ ? 4u * H.n_sel * 32u : 0u;
        if (ch_smem_ && 16u * 4u * H.n_sel + 4u * (H.off_inputs - H.off_thr) > 60u * 1024u) {
            *why = "the selection thresholds exceed constant memory";
            return false;
        }
        out->dyn_smem = ch_smem_ ? ch_off + ch_bytes : 0u;
        /* SA, SB, PF, ZF and the barrier */
        out->static_smem = 2u * 4u * 32u * H.W32 + 4u * 4u * 32u + 256u;
        if ((out->dyn_smem ? out->dyn_smem : (tab_smem ? table_bytes : 0u)) + out->static_smem >
            227u * 1024u) { /* opt-in shared memory of a CTA on sm_103a */
            *why = "the states, tables and choices exceed the shared memory of a CTA";
            return false;
        }
        Pv = H.P;
        hmax = Pv ? (31u - (uint32_t)__builtin_ctz(Pv)) / 2u + 1u : 0u;
        const uint32_t npairs = (H.W32 + 1) / 2; /* row pairs: one uint64 state word each */
        /* groups by output row, and the cost of each row pair */
        const uint32_t* wgroups = V.at<uint32_t>(H.off_wgroups);
        std::vector<std::vector<uint32_t>> row_groups(H.W32);
        for (uint32_t r = 0; r < H.W32; ++r)
            for (uint32_t i = words[r].x; i < words[r].x + words[r].y; ++i) row_groups[r].push_back(wgroups[i]);
        std::vector<double> cost(npairs, 0.0);
        double total = 0;
        for (uint32_t r = 0; r < H.W32; ++r)
            for (uint32_t g : row_groups[r]) {
                const double c = 8.0 + 3.0 * groups[g].q + 12.0 * groups[g].n_mul;
                cost[r / 2] += c;
                total += c;
            }
        /* two warps per CTA unless asked: on the scale-free network 2 warps ran faster
         * than 1, 3, 4 or 8 (more warps add barrier waits and re-drawn SEL blocks,
         * fewer leave too little to overlap) */
        uint32_t K = (flags_ >> 8) & 31u;
        if (!K) K = 2;
        (void)total;
        K = std::max(1u, std::min(K, npairs));
        warps = K;
        /* row pairs to warps: largest first to the least loaded warp */
        std::vector<uint32_t> order(npairs);
        for (uint32_t i = 0; i < npairs; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
        std::vector<double> load(K, 0.0);
        std::vector<std::vector<uint32_t>> pairs_of(K);
        for (uint32_t pr : order) {
            const uint32_t w = (uint32_t)(std::min_element(load.begin(), load.end()) - load.begin());
            pairs_of[w].push_back(pr);
            load[w] += cost[pr] + 1.0;
        }
        for (auto& v : pairs_of) std::sort(v.begin(), v.end());
        const uint32_t wpairs = (H.W + 1) / 2; /* perturbation word pairs, round robin */

        o << "#include \"pbn_device.cuh\"\n";
        if (geometric) {
            const uint64_t* G = V.at<uint64_t>(H.off_geo);
            o << "__device__ const unsigned long long GEO_T[64] = {";
            for (int k = 0; k < 64; ++k) o << (k ? ", " : "") << fmt("0x%016llxull", (unsigned long long)G[k]);
            o << "};\n";
        }
        const uint32_t R = H.W32;
        if (ch_smem_) {
            /* per SEL slot (4 per block, slot-major): t1, t2, number of thresholds, first
             * extra threshold; the block counters; the extra thresholds */
            o << "__constant__ uint4 SELS[" << 4 * H.n_sel << "] = {";
            for (uint32_t slot = 0; slot < 4 * H.n_sel; ++slot) {
                const uint32_t* ss = selslot + 4 * ((slot & 3u) * H.n_sel + (slot >> 2));
                o << (slot ? (slot % 4 ? ", " : ",\n  ") : "") << "{" << hex32(ss[0]) << ", " << hex32(ss[1]) << ", "
                  << ss[2] << "u, " << ss[3] << "u}";
            }
            o << "};\n__constant__ uint32_t SELB[" << H.n_sel << "] = {";
            for (uint32_t b = 0; b < H.n_sel; ++b) o << (b ? ", " : "") << hex32((PBN_DOM_SEL << 28) | selblk[b]);
            const uint32_t nthr = std::max<uint32_t>(1u, (H.off_inputs - H.off_thr) / 4u);
            o << "};\n__constant__ uint32_t SELT[" << nthr << "] = {";
            for (uint32_t i = 0; i < nthr; ++i) o << (i ? (i % 8 ? ", " : ",\n  ") : "") << hex32(i < (H.off_inputs - H.off_thr) / 4u ? thr[i] : 0u);
            o << "};\n";
        }
        const uint32_t minctas = (flags_ >> 13) & 7u; /* resident CTAs per SM the registers must allow */
        o << "extern \"C\" __global__ void __launch_bounds__(" << 32 * K;
        if (minctas) o << ", " << minctas;
        o << ") pbn_plan_kernel(const pbn_jit_params P) {\n"
             "  extern __shared__ __align__(128) uint8_t smem[];\n  __shared__ __align__(8) uint64_t bar;\n"
          << "  __shared__ uint32_t SA[" << R * 32 << "], SB[" << R * 32 << "];\n"
             "  __shared__ uint32_t PF[2][32], ZF[2][32];\n";
        if (tab_smem) {
            o << "  if (!pbn_stage(smem, P.image + P.off_tables, P.tab_bytes, &bar)) {\n"
                 "    if (threadIdx.x == 0 && P.status) atomicOr(P.status, 1u);\n    return;\n  }\n"
                 "  const uint32_t* TAB = reinterpret_cast<const uint32_t*>(smem);\n";
        } else {
            o << "  const uint32_t* __restrict__ TAB = reinterpret_cast<const uint32_t*>(P.image + P.off_tables);\n";
        }
        o << "  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;\n"
             "  const uint32_t lt = blockIdx.x * 32u + lane;\n"
             "  const bool active = lt < P.n_traj;\n"
             "  const uint64_t traj = P.traj_begin + lt;\n"
             "  uint32_t cV = 0, c01 = 0, c10 = 0, c11 = 0;\n";
        if (ch_smem_)
            o << "  uint8_t* const CH = smem + " << ch_off << "u; /* [slot][lane] choice bytes */\n"
                 "  const uint8_t* const CHs = CH + lane;\n";
        o << ""
          << "  for (uint32_t i = threadIdx.x; i < " << R * 32 << "u; i += blockDim.x) SA[i] = 0u;\n"
             "  for (uint32_t i = threadIdx.x; i < 64u; i += blockDim.x) { PF[i >> 5][i & 31u] = 0u; ZF[i >> 5][i & 31u] = 1u; }\n"
             "  __syncthreads();\n";
        /* initial state: keyed (INIT word pairs round robin, bits ORed into the rows) or
         * loaded (each warp its own row pairs) */
        o << "  if (P.init == 0) {\n    const pbn_philox_step ps0 = pbn_philox_begin(P, traj, 0);\n    switch (warp) {\n";
        for (uint32_t w = 0; w < K; ++w) {
            o << "    case " << w << "u: {\n";
            for (uint32_t pr = w; 2 * pr < H.W; pr += K) {
                const uint64_t r0 = ret[2 * pr], r1 = (2 * pr + 1 < H.W) ? ret[2 * pr + 1] : 0;
                if (!(r0 | r1)) continue;
                o << "      { const uint4 I = pbn_philox_draw(P, ps0, " << hex32((PBN_DOM_INIT << 28) | pr) << ");\n";
                /* the bits of each target row, then one atomic OR per row */
                std::map<uint32_t, std::string> rows;
                for (uint32_t half = 0; half < 2; ++half) {
                    const uint32_t wd = 2 * pr + half;
                    const uint64_t rw = half ? r1 : r0;
                    for (uint32_t b = 0; b < 64; ++b) {
                        if (!((rw >> b) & 1u)) continue;
                        const uint32_t ps = pos[64 * wd + b];
                        const char comp = lanes[2 * half + (b >= 32 ? 1 : 0)];
                        std::string& e = rows[ps >> 5];
                        e += (e.empty() ? "" : " | ") + fmt("(((I.%c >> %u) & 1u) << %u)", comp, b & 31, ps & 31);
                    }
                }
                for (const auto& kv : rows)
                    o << "        atomicOr(&SA[" << kv.first << "u * 32u + lane], " << kv.second << ");\n";
                o << "      }\n";
            }
            o << "    } break;\n";
        }
        o << "    default: break;\n    }\n  } else if (active) {\n    switch (warp) {\n";
        for (uint32_t w = 0; w < K; ++w) {
            o << "    case " << w << "u:\n";
            for (uint32_t pr : pairs_of[w]) {
                o << "      { const uint64_t v = P.state[(uint64_t)" << pr << " * P.n_traj + lt]; SA[" << 2 * pr
                  << "u * 32u + lane] = (uint32_t)v;";
                if (2 * pr + 1 < R) o << " SA[" << 2 * pr + 1 << "u * 32u + lane] = (uint32_t)(v >> 32);";
                o << " }\n";
            }
            o << "      break;\n";
        }
        o << "    default: break;\n    }\n  }\n  __syncthreads();\n";
        /* meta-state indicator of s(step_begin): warp 0, every row */
        o << "  uint32_t zp = 1u;\n  if (warp == 0) {\n";
        for (uint32_t r = 0; r < R; ++r)
            o << "    zp &= (uint32_t)((SA[" << r << "u * 32u + lane] & P.meta_mask[" << r << "]) == P.meta_val[" << r
              << "]);\n";
        o << "    if (P.count_first) cV += zp;\n  }\n";
        o << "  for (uint32_t k = 0; k < P.n_steps; ++k) {\n"
             "    const uint64_t t = P.step_begin + k;\n"
             "    const pbn_philox_step ps = pbn_philox_begin(P, traj, t);\n"
             "    uint32_t* const Sc = (k & 1u) ? SB : SA;\n"
             "    uint32_t* const Sn = (k & 1u) ? SA : SB;\n"
             "    if (warp == 0) {\n"
             "      PF[(k + 1u) & 1u][lane] = 0u;\n"
             "      if (k > 0) { /* counts of the state the previous step produced */\n"
             "        const uint32_t z = ZF[(k + 1u) & 1u][lane];\n"
             "        ZF[(k + 1u) & 1u][lane] = 1u;\n"
             "        const uint32_t kk = k - 1u;\n"
             "        const uint32_t cv = kk >= P.kv0 ? 1u : 0u, cp = kk >= P.kp0 ? 1u : 0u;\n"
             "        cV += cv & z; c11 += cp & zp & z; c01 += cp & (zp ^ 1u) & z; c10 += cp & zp & (z ^ 1u); zp = z;\n"
             "      }\n    }\n";
        /* phase A: perturbation word pairs round robin over the warps */
        o << "    switch (warp) {\n";
        for (uint32_t w = 0; w < K; ++w) {
            o << "    case " << w << "u: {\n      uint32_t any = 0;\n";
            pair_sel_.assign(wpairs, 0);
            bool anyw = false;
            for (uint32_t pr = w; pr < wpairs; pr += K) pair_sel_[pr] = 1, anyw = true;
            if (Pv && anyw) {
                if (geometric) emit_geometric_perturbation("@", "");
                else emit_paired_perturbation("@", "");
            }
            o << "      if (any) PF[k & 1u][lane] = 1u;\n    } break;\n";
        }
        pair_sel_.clear();
        o << "    default: break;\n    }\n";
        if (ch_smem_)
            o << "    /* the SEL blocks, round robin over the warps: choices as bytes */\n"
                 "#pragma unroll 1\n"
                 "    for (uint32_t b = warp; b < " << H.n_sel << "u; b += " << K << "u) {\n"
                 "      const uint4 x = pbn_philox_draw(P, ps, SELB[b]);\n"
                 "      const uint32_t u[4] = {x.x, x.y, x.z, x.w};\n"
                 "#pragma unroll\n"
                 "      for (int l = 0; l < 4; ++l) {\n"
                 "        const uint4 S = SELS[4u * b + l];\n"
                 "        uint32_t j = ((S.z >= 1u) & (u[l] >= S.x)) + ((S.z >= 2u) & (u[l] >= S.y));\n"
                 "        if (S.z > 2u) { j = 0; for (uint32_t q = 0; q < S.z; ++q) j += (u[l] >= SELT[S.w + q]) ? 1u : 0u; }\n"
                 "        CH[(4u * b + l) * 32u + lane] = (uint8_t)j;\n"
                 "      }\n    }\n";
        o << "    __syncthreads();\n"
             "    const uint32_t pert = PF[k & 1u][lane];\n"
             "    const uint32_t scb = (uint32_t)__cvta_generic_to_shared(Sc) + 4u * lane;\n";
        /* phase B: each warp's row pairs */
        o << "    switch (warp) {\n";
        for (uint32_t w = 0; w < K; ++w) {
            o << "    case " << w << "u: {\n";
            std::vector<uint32_t> myrows;
            for (uint32_t pr : pairs_of[w]) {
                myrows.push_back(2 * pr);
                if (2 * pr + 1 < R) myrows.push_back(2 * pr + 1);
            }
            for (uint32_t r : myrows) o << "      uint32_t n" << r << " = 0;\n";
            o << "      if (!pert) {\n";
            /* the rows' groups in the order of the last SEL block they read; each block
             * drawn before its first use, each state row loaded before its first use */
            std::vector<std::pair<uint32_t, uint32_t>> order2;
            for (uint32_t r : myrows)
                for (uint32_t g : row_groups[r]) order2.push_back({r, g});
            std::stable_sort(order2.begin(), order2.end(), [&](const std::pair<uint32_t, uint32_t>& x,
                                                               const std::pair<uint32_t, uint32_t>& y) {
                const auto bx = blocks_of(x.second), by = blocks_of(y.second);
                const uint32_t mx = bx.empty() ? 0 : *std::max_element(bx.begin(), bx.end());
                const uint32_t my = by.empty() ? 0 : *std::max_element(by.begin(), by.end());
                return mx < my;
            });
            /* a block drawn more than kReuse groups earlier is drawn again (a new
             * version of its choices), so that no choice stays live for long */
            const uint32_t kReuse = (uint32_t)ws_reuse;
            std::vector<int64_t> drawn_at(H.n_sel, -1);
            std::vector<uint32_t> version(H.n_sel, 0);
            int64_t gcount = 0;
            /* groups in batches: the SEL blocks of a batch are drawn, then the state rows
             * its groups read are loaded together, then the groups are evaluated, so
             * that a batch's loads and lookups are in flight at once */
            const uint32_t batch = 1u << (2u * ((flags_ >> 16) & 3u)); /* 1, 4, 16, 64 */
            for (size_t b0 = 0; b0 < order2.size(); b0 += batch) {
              const size_t b1 = std::min(order2.size(), b0 + (size_t)batch);
              for (size_t bi = b0; bi < b1; ++bi) {
                const uint32_t gi = order2[bi].second;
                for (uint32_t b : blocks_of(gi))
                    if (!ch_smem_ && (drawn_at[b] < 0 || gcount - drawn_at[b] > (int64_t)kReuse)) {
                        /* the block's four uniforms become the choices of its slots at once
                         * (one register per node instead of four per block) */
                        drawn_at[b] = gcount;
                        if (++version[b] == 1) { /* declared at the first draw, assigned at each */
                            bool first = true;
                            for (uint32_t l = 0; l < 4; ++l) {
                                if (slot_choice(4 * b + l).empty()) continue;
                                o << (first ? "        uint32_t " : ", ") << "J" << 4 * b + l;
                                first = false;
                            }
                            if (!first) o << ";\n";
                        }
                        o << "        { const uint4 U" << b << " = pbn_philox_draw(P, ps, "
                          << hex32((PBN_DOM_SEL << 28) | selblk[b]) << ");";
                        for (uint32_t l = 0; l < 4; ++l) {
                            const std::string j = slot_choice(4 * b + l);
                            if (!j.empty()) o << " J" << 4 * b + l << " = " << j << ";";
                        }
                        o << " }\n";
                    }
                ++gcount;
              }
              /* the batch's input rows, loaded in its own scope (volatile shared loads
               * are not merged across batches, so no row stays live in a register for
               * the rest of the warp's code) */
              std::vector<uint32_t> brows;
              for (size_t bi = b0; bi < b1; ++bi)
                  for (uint32_t row : rows_read(order2[bi].second))
                      if (row < R) brows.push_back(row);
              std::sort(brows.begin(), brows.end());
              brows.erase(std::unique(brows.begin(), brows.end()), brows.end());
              o << "        { ";
              for (uint32_t row : brows)
                  o << "uint32_t s" << row << "; asm volatile(\"ld.shared.u32 %0, [%1+" << row * 128
                    << "];\" : \"=r\"(s" << row << ") : \"r\"(scb)); ";
              o << "\n";
              for (size_t bi = b0; bi < b1; ++bi) {
                  const uint32_t r = order2[bi].first, gi = order2[bi].second;
                  const pbn_img_group& G = groups[gi];
                  o << "          { ";
                  if (G.l2w == PBN_IMG_SPLIT) emit_split_group(r, G);
                  else emit_merged_group(r, gi, G);
              }
              o << "        }\n";
            }
            o << "      } else {\n";
            for (uint32_t r : myrows) o << "        n" << r << " = Sc[" << r << "u * 32u + lane];\n";
            o << "      }\n";
            for (uint32_t r : myrows) o << "      Sn[" << r << "u * 32u + lane] = n" << r << ";\n";
            /* this warp's part of the meta-state indicator of the new state */
            o << "      if (";
            for (size_t i = 0; i < myrows.size(); ++i)
                o << (i ? " || " : "") << "((n" << myrows[i] << " & P.meta_mask[" << myrows[i] << "]) != P.meta_val["
                  << myrows[i] << "])";
            o << ") ZF[k & 1u][lane] = 0u;\n";
            /* trace: this warp's row pairs of the new state */
            o << "      if (P.trace && active && (k + 1) % P.trace_stride == 0) {\n"
                 "        const uint64_t snap = (k + 1) / P.trace_stride - 1;\n";
            for (uint32_t pr : pairs_of[w])
                o << "        P.trace[(snap * " << npairs << "u + " << pr << "u) * P.n_traj + lt] = ((uint64_t)"
                  << (2 * pr + 1 < R ? "n" + std::to_string(2 * pr + 1) : std::string("0u")) << " << 32) | n" << 2 * pr
                  << ";\n";
            o << "      }\n    } break;\n";
        }
        o << "    default: break;\n    }\n    __syncthreads();\n  }\n";
        /* the last step's counts, the final state and the pooled counts */
        o << "  if (warp == 0 && P.n_steps > 0) {\n"
             "    const uint32_t z = ZF[(P.n_steps + 1u) & 1u][lane];\n"
             "    const uint32_t kk = P.n_steps - 1u;\n"
             "    const uint32_t cv = kk >= P.kv0 ? 1u : 0u, cp = kk >= P.kp0 ? 1u : 0u;\n"
             "    cV += cv & z; c11 += cp & zp & z; c01 += cp & (zp ^ 1u) & z; c10 += cp & zp & (z ^ 1u);\n"
             "  }\n"
             "  const uint32_t* const Sf = (P.n_steps & 1u) ? SB : SA;\n"
             "  if (active) {\n    switch (warp) {\n";
        for (uint32_t w = 0; w < K; ++w) {
            o << "    case " << w << "u:\n";
            for (uint32_t pr : pairs_of[w]) {
                o << "      P.state[(uint64_t)" << pr << " * P.n_traj + lt] = ";
                if (2 * pr + 1 < R) o << "((uint64_t)Sf[" << 2 * pr + 1 << "u * 32u + lane] << 32) | ";
                o << "Sf[" << 2 * pr << "u * 32u + lane];\n";
            }
            o << "      break;\n";
        }
        o << "    default: break;\n    }\n"
             "    if (warp == 0 && P.counts) {\n"
             "      const uint64_t nt = P.n_traj;\n"
             "      P.counts[lt] += cV; P.counts[nt + lt] += P.pairs - c01 - c10 - c11;\n"
             "      P.counts[2 * nt + lt] += c01; P.counts[3 * nt + lt] += c10; P.counts[4 * nt + lt] += c11;\n"
             "    }\n  }\n";
        o << "  if (warp == 0 && P.pooled) {\n"
             "    uint64_t v[5] = {active ? cV : 0u, active ? (uint64_t)(P.pairs - c01 - c10 - c11) : 0u,\n"
             "                     active ? c01 : 0u, active ? c10 : 0u, active ? c11 : 0u};\n"
             "#pragma unroll\n    for (int i = 0; i < 5; ++i) {\n"
             "#pragma unroll\n      for (int d = 16; d > 0; d >>= 1) v[i] += __shfl_xor_sync(0xFFFFFFFFu, v[i], d);\n    }\n"
             "    if (lane == 0) {\n"
             "      for (int i = 0; i < 5; ++i) if (v[i]) atomicAdd(P.pooled + i, (unsigned long long)v[i]);\n    }\n  }\n";
        o << "}\n";
        out->src = o.str();
        out->warps = K;
        return true;
    }

    /* state rows a group's input bits come from */
    std::vector<uint32_t> rows_read(uint32_t gi) const {
        std::vector<uint32_t> rows;
        const pbn_img_group& G = groups[gi];
        auto add = [&](uint32_t in_chunk, uint32_t k, uint32_t stride) {
            for (uint32_t b = 0; b < k; ++b) rows.push_back(inrec[4 * (in_chunk + stride * (b / 4)) + (b & 3)] >> 7);
        };
        if (G.l2w == PBN_IMG_SPLIT) {
            for (uint32_t f = 0; f < G.q; ++f) {
                const uint32_t* F = subs + 2 * (G.tab_off + 32 * f);
                add(F[0] & 0x7FFFFFFu, F[0] >> 27, 1);
            }
        } else {
            add(G.in_chunk, G.q, 32);
        }
        std::sort(rows.begin(), rows.end());
        rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
        return rows;
    }

public:
    uint32_t warps = 0; /* warps per CTA of the warp-split form (0: one trajectory per thread) */

private:
    /* a group that gathers some of its inputs by multiplication (PBN_COMPILE_MAGIC_GATHER) */
    struct GTerm {
        bool magic;
        MagicTerm m;         /* magic == true */
        uint32_t row, bit;   /* single bit */
        uint32_t off;        /* position of the field in the new index */
    };
    struct GPlan {
        bool used = false;
        std::vector<GTerm> terms;
        uint32_t qn = 0, tab_off = 0, tab_words = 0;
    };

    const pbn_img_header& H;
    View V;
    const uint32_t flags_;
    const bool wide; /* SEL blocks drawn lazily in group order: their uniforms live only
                        while the groups that need them are evaluated */
    const BatchSpec* bs_; /* batch-module function instead of a kernel */
    std::vector<uint8_t> pair_sel_; /* warp split: the perturbation word pairs one warp draws (empty: all) */
    bool pair_selected(uint32_t wp) const { return pair_sel_.empty() || (wp < pair_sel_.size() && pair_sel_[wp]); }
    const std::string sfx_; /* suffix of the module-level names (unique per network) */
    bool ws_choices_ = false; /* choices as J<slot> registers computed after each draw */
    bool ch_smem_ = false;    /* choices as bytes CH[slot][lane] in shared memory */
  public:
    int ws_reuse = 16;        /* warp split: groups over which a drawn SEL block is reused */
  private:
    const uint2* words = nullptr;
    const pbn_img_group* groups = nullptr;
    const pbn_img_multi* multi = nullptr;
    const uint32_t *thr = nullptr, *inrec = nullptr, *selblk = nullptr, *pos = nullptr, *tab = nullptr;
    const uint32_t *selslot = nullptr, *subs = nullptr;
    const uint64_t* ret = nullptr;
    uint32_t table_bytes = 0;
    std::vector<uint32_t> tab_starts; /* start offsets of every table, sorted */
    std::vector<GPlan> gp;
    std::vector<uint32_t> tabm;       /* the plan's tables, then the rebuilt ones */
    bool magic = false, tab_smem = false;
    bool geometric = false, pipelined = false, interleave = false, nodewise = false;
    uint32_t Pv = 0, hmax = 0;
    std::string z; /* meta-state indicator of s */
    std::ostringstream o;

    bool fits(std::string* why) const {
        if (H.W32 > 64) {
            *why = "state wider than 64 words";
            return false;
        }
        if (H.W > (wide ? 32u : 16u)) {
            *why = wide ? "more than 2048 original nodes" : "more than 1024 original nodes";
            return false;
        }
        if (!wide && H.n_sel > 24) {
            *why = "more than 24 selection blocks per step";
            return false;
        }
        return true;
    }

    void bind_sections() {
        words = V.at<uint2>(H.off_words);
        groups = V.at<pbn_img_group>(H.off_groups);
        multi = V.at<pbn_img_multi>(H.off_multi);
        thr = V.at<uint32_t>(H.off_thr);
        inrec = V.at<uint32_t>(H.off_inputs);
        selblk = V.at<uint32_t>(H.off_selblk);
        ret = V.at<uint64_t>(H.off_ret);
        pos = V.at<uint32_t>(H.off_pos);
        tab = V.at<uint32_t>(H.off_tables);
        table_bytes = H.off_ret - H.off_tables;
        selslot = V.at<uint32_t>(H.off_selslot);
        subs = V.at<uint32_t>(H.off_subs);
    }

    /* start offsets of every table (merged groups and split-node functions), sorted */
    void collect_table_starts() {
        for (uint32_t g = 0; g < H.n_groups; ++g) {
            if (groups[g].l2w != PBN_IMG_SPLIT) tab_starts.push_back(groups[g].tab_off);
            else
                for (uint32_t f = 0; f < groups[g].q; ++f) tab_starts.push_back(subs[2 * (groups[g].tab_off + 32 * f) + 1]);
        }
        std::sort(tab_starts.begin(), tab_starts.end());
    }

    /* Multiply gathers (PBN_COMPILE_MAGIC_GATHER): for every merged group, the inputs
     * of one state word with 3 to 8 bits become one multiply-gather field when an
     * injective multiplier exists; the other inputs stay single-bit gathers.  Such a
     * group gets its table rebuilt in the new index order, appended after a copy of
     * the plan's tables; the kernel then reads its tables from that array (a
     * __device__ array of the generated source) instead of the plan image. */
    void plan_multiply_gathers() {
        gp.assign(H.n_groups, GPlan{});
        magic = (flags_ & PBN_COMPILE_MAGIC_GATHER) != 0 && table_bytes <= 256u * 1024u;
        if (!magic) return;
        tabm.assign(tab, tab + table_bytes / 4);
        for (uint32_t g = 0; g < H.n_groups; ++g) {
            const pbn_img_group& G = groups[g];
            if (G.l2w == PBN_IMG_SPLIT || G.q < 3) continue;
            std::vector<uint32_t> rowb(G.q), bitb(G.q);
            for (uint32_t b = 0; b < G.q; ++b) {
                const uint32_t rec = inrec[4 * (G.in_chunk + 32 * (b / 4)) + (b & 3)];
                rowb[b] = rec >> 7;
                bitb[b] = ((b & 3) + (rec & 31)) & 31;
            }
            std::vector<uint32_t> rows(rowb);
            std::sort(rows.begin(), rows.end());
            rows.erase(std::unique(rows.begin(), rows.end()), rows.end());
            GPlan GP;
            uint32_t off = 0;
            bool any = false;
            for (uint32_t r : rows) {
                std::vector<uint32_t> a;
                for (uint32_t b = 0; b < G.q; ++b)
                    if (rowb[b] == r) a.push_back(bitb[b]);
                std::sort(a.begin(), a.end());
                MagicTerm m;
                if (find_magic(r, a, &m)) {
                    GP.terms.push_back(GTerm{true, m, r, 0, off});
                    off += m.width;
                    any = true;
                } else {
                    for (uint32_t x : a) GP.terms.push_back(GTerm{false, MagicTerm{}, r, x, off++});
                }
            }
            if (!any || off > 24) continue;
            /* combined choices held by the table (padding entries are zero) */
            auto nx = std::upper_bound(tab_starts.begin(), tab_starts.end(), G.tab_off);
            const uint64_t words_old = (nx == tab_starts.end() ? table_bytes / 4 : *nx) - G.tab_off;
            const uint64_t prod = std::max<uint64_t>(1, (words_old * 32) >> (G.q + G.l2w));
            const uint64_t bits_new = (prod << off) << G.l2w;
            /* the copy plus the rebuilt tables stay within what is staged in shared memory */
            if (bits_new > (UINT64_C(1) << 24) || (tabm.size() + (bits_new + 31) / 32) * 4 > 48u * 1024u) continue;
            GP.tab_off = (uint32_t)tabm.size();
            GP.tab_words = (uint32_t)((bits_new + 31) / 32);
            tabm.resize(tabm.size() + GP.tab_words, 0u);
            uint32_t* dst = tabm.data() + GP.tab_off;
            const uint32_t emask = G.l2w >= 5 ? 0xFFFFFFFFu : ((1u << (1u << G.l2w)) - 1u);
            for (uint64_t c = 0; c < prod; ++c) {
                for (uint32_t x = 0; x < (1u << G.q); ++x) {
                    const uint64_t bo = ((c << G.q) | x) << G.l2w;
                    if ((bo >> 5) >= words_old) continue;
                    const uint32_t v = (tab[G.tab_off + (bo >> 5)] >> (bo & 31)) & emask;
                    /* the input pattern x as state words, then its new index */
                    std::vector<uint32_t> sw(H.W32, 0u);
                    for (uint32_t b = 0; b < G.q; ++b) sw[rowb[b]] |= ((x >> b) & 1u) << bitb[b];
                    uint32_t xn = 0;
                    for (const GTerm& t : GP.terms)
                        xn |= (t.magic ? magic_field(t.m, sw[t.m.row]) : ((sw[t.row] >> t.bit) & 1u)) << t.off;
                    const uint64_t bn = ((c << off) | xn) << G.l2w;
                    dst[bn >> 5] |= v << (bn & 31);
                }
            }
            GP.used = true;
            GP.qn = off;
            gp[g] = std::move(GP);
        }
        tabm.resize((tabm.size() + 3) & ~(size_t)3, 0u); /* bulk copies move multiples of 16 bytes */
        table_bytes = (uint32_t)(tabm.size() * 4);
    }

    /* the geometric sampler's thresholds and the rebuilt tables, as __device__ arrays */
    void emit_globals() {
        if (!bs_) o << "#include \"pbn_device.cuh\"\n";
        if (H.sampler == PBN_PERT_GEOMETRIC) {
            const uint64_t* G = V.at<uint64_t>(H.off_geo);
            o << "__device__ const unsigned long long GEO_T" << sfx_ << "[64] = {";
            for (int k = 0; k < 64; ++k) o << (k ? ", " : "") << fmt("0x%016llxull", (unsigned long long)G[k]);
            o << "};\n";
        }
        if (magic) {
            /* the plan's tables followed by the rebuilt tables of multiply-gather groups */
            o << "__device__ __align__(16) const uint32_t TABM[" << std::max<size_t>(tabm.size(), 4) << "] = {";
            for (size_t i = 0; i < tabm.size(); ++i) o << (i ? (i % 8 ? ", " : ",\n  ") : "") << hex32(tabm[i]);
            o << "};\n";
        }
    }

    /* kernel entry, table staging, the initial state (keyed INIT draws or the stored
     * state) and the meta-state indicator of s(step_begin) */
    void emit_prologue() {
        if (bs_) return emit_batch_prologue();
        const char* tab_src = magic ? "reinterpret_cast<const uint8_t*>(TABM)" : "P.image + P.off_tables";
        o << "extern \"C\" __global__ void __launch_bounds__(512) pbn_plan_kernel(const pbn_jit_params P) {\n";
        o << "  extern __shared__ __align__(128) uint8_t smem[];\n  __shared__ __align__(8) uint64_t bar;\n";
        if (tab_smem) {
            o << "  if (!pbn_stage(smem, " << tab_src << ", P.tab_bytes, &bar)) {\n"
                 "    if (threadIdx.x == 0 && P.status) atomicOr(P.status, 1u);\n    return;\n  }\n"
                 "  const uint32_t* TAB = reinterpret_cast<const uint32_t*>(smem);\n";
        } else {
            o << "  const uint32_t* __restrict__ TAB = reinterpret_cast<const uint32_t*>(" << tab_src << ");\n";
        }
        o << "  const uint32_t lt = blockIdx.x * blockDim.x + threadIdx.x;\n"
             "  const bool active = lt < P.n_traj;\n";
        emit_initial_state();
    }

    /* Batch-module function of one work item: the launch fields come from the
     * network's descriptor and the launch, the keys are literals (immediates once the
     * aggregate is scalarised), the tables are read from the staged shared memory or
     * the plan image, one trajectory per thread of the item. */
    void emit_batch_prologue() {
        const uint64_t seed = bs_->seed;
        const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
        o << "extern \"C\" __device__ __noinline__ bool pbn_net" << sfx_
          << "(const pbn_netdesc& D, const pbn_workitem W, const uint64_t step_offset, const uint32_t n_steps, "
             "uint32_t* cnt, const uint8_t* kernel_smem, uint32_t* status) {\n";
        o << "  extern __shared__ __align__(128) uint8_t smem[];\n"
             "  if (static_cast<const uint8_t*>(smem) != kernel_smem) {\n"
             "    if (status) atomicOr(status, PBN_BATCH_BAD_MODULE);\n    return false;\n  }\n";
        o << "  const pbn_item_window w = pbn_item_window_at(D, step_offset, n_steps);\n";
        o << "  struct PV { uint32_t key0[10], key1[10]; uint64_t* state; uint64_t* counts; uint64_t* trace;\n"
             "    uint32_t trace_stride; uint64_t traj_begin, step_begin;\n"
             "    uint32_t n_traj, n_steps, kv0, kp0, pairs, count_first, init; };\n";
        o << "  const PV P = {{";
        for (int r = 0; r < 10; ++r) o << (r ? ", " : "") << hex32(k0 + (uint32_t)r * 0x9E3779B9u);
        o << "}, {";
        for (int r = 0; r < 10; ++r) o << (r ? ", " : "") << hex32(k1 + (uint32_t)r * 0xBB67AE85u);
        o << "},\n    D.state, D.counts, nullptr, 1u, D.traj_begin, w.step_begin,\n"
             "    D.n_traj, w.n_steps, w.kv0, w.kp0, w.pairs, w.count_first, w.init};\n";
        if (tab_smem) o << "  const uint32_t* TAB = reinterpret_cast<const uint32_t*>(smem);\n";
        else
            o << "  const uint32_t* __restrict__ TAB = reinterpret_cast<const uint32_t*>(D.image + " << H.off_tables
              << "u);\n";
        o << "  const uint32_t lt = W.t0 + threadIdx.x;\n"
             "  const bool active = threadIdx.x < W.n;\n";
        emit_initial_state();
    }

    /* the counters, the initial state (keyed INIT draws or the stored state) and the
     * meta-state indicator of s(step_begin) */
    void emit_initial_state() {
        o << "  const uint64_t traj = P.traj_begin + lt;\n"
             "  uint32_t cV = 0, c01 = 0, c10 = 0, c11 = 0;\n";
        o << "  uint32_t";
        for (uint32_t r = 0; r < H.W32; ++r) o << (r ? ", " : " ") << "s" << r << " = 0";
        o << ";\n  if (active) {\n";
        /* initial state */
        o << "    if (P.init == 0) {\n      const pbn_philox_step ps = pbn_philox_begin(P, traj, 0);\n";
        for (uint32_t pr = 0; 2 * pr < H.W; ++pr) {
            const uint64_t r0 = ret[2 * pr], r1 = (2 * pr + 1 < H.W) ? ret[2 * pr + 1] : 0;
            if (!(r0 | r1)) continue;
            o << "      const uint4 I" << pr << " = pbn_philox_draw(P, ps, " << hex32((PBN_DOM_INIT << 28) | pr) << ");\n";
            for (uint32_t half = 0; half < 2; ++half) {
                const uint32_t w = 2 * pr + half;
                const uint64_t rw = half ? r1 : r0;
                for (uint32_t b = 0; b < 64; ++b) {
                    if (!((rw >> b) & 1u)) continue;
                    const uint32_t ps = pos[64 * w + b], row = ps >> 5, bit = ps & 31;
                    const char comp = lanes[2 * half + (b >= 32 ? 1 : 0)];
                    o << fmt("      s%u |= ((I%u.%c >> %u) & 1u) << %u;\n", row, pr, comp, b & 31, bit);
                }
            }
        }
        o << "    } else {\n";
        for (uint32_t r = 0; r < H.W32; r += 2)
            o << "      { const uint64_t v = P.state[(uint64_t)" << r / 2 << " * P.n_traj + lt]; s" << r
              << " = (uint32_t)v; s" << r + 1 << " = (uint32_t)(v >> 32); }\n";
        o << "    }\n";
        std::ostringstream zs;
        zs << "(";
        if (bs_) {
            /* the network's meta-state rows as immediates */
            for (uint32_t m = 0; m < bs_->meta.n_rows; ++m)
                zs << (m ? " & " : "") << "(uint32_t)((s" << bs_->meta.row[m] << " & " << hex32(bs_->meta.mask[m])
                   << ") == " << hex32(bs_->meta.val[m]) << ")";
            if (!bs_->meta.n_rows) zs << "1u";
        } else {
            for (uint32_t r = 0; r < H.W32; ++r)
                zs << (r ? " & " : "") << "(uint32_t)((s" << r << " & P.meta_mask[" << r << "]) == P.meta_val[" << r
                   << "])";
        }
        zs << ")";
        z = zs.str();
        o << "    uint32_t zp = " << z << ";\n    if (P.count_first) cV += zp;\n";
    }

    /* the SEL blocks of one step as uint4 <name><i> drawn from Philox state <ps> */
    void emit_sel_draws(const char* ind, const char* decl, const char* name, const char* ps) {
        for (uint32_t i = 0; i < H.n_sel; ++i)
            o << ind << decl << name << i << " = pbn_philox_draw(P, " << ps << ", "
              << hex32((PBN_DOM_SEL << 28) | selblk[i]) << ");\n";
    }

    /* perturbed retained lanes of word w (masks pl/ph): op into s<row> or a mask */
    void emit_flips(uint32_t w, const std::string& pl, const std::string& ph, const char* target, const char* op) {
        const uint32_t rl = (uint32_t)ret[w], rh = (uint32_t)(ret[w] >> 32);
        for (int half = 0; half < 2; ++half) {
            const uint32_t rm = half ? rh : rl;
            if (!rm) continue;
            o << "          { uint32_t f = " << (half ? ph : pl) << " & " << hex32(rm) << ";\n"
              << "          while (f) { const uint32_t b = __ffs(f) - 1; f &= f - 1; switch (b) {\n";
            for (uint32_t b = 0; b < 32; ++b) {
                if (!((rm >> b) & 1u)) continue;
                const uint32_t ps = pos[64 * w + 32 * half + b];
                if (target[0] == '@') /* warp split: the flip goes to the shared state word */
                    o << "            case " << b << ": atomicXor(&Sc[" << (ps >> 5) << "u * 32u + lane], "
                      << hex32(1u << (ps & 31)) << "); break;\n";
                else
                    o << "            case " << b << ": " << target << (ps >> 5) << " " << op << " "
                      << hex32(1u << (ps & 31)) << "; break;\n";
            }
            o << "          } } }\n";
        }
    }

    /* lanes of original word w that hold nodes */
    uint64_t valid_of(uint32_t w) const {
        const uint32_t nl = (w == H.W - 1) ? (H.n - 64 * w) : 64u;
        return nl >= 64 ? ~0ull : ((1ull << nl) - 1ull);
    }

    /* one straight-line level pair h of word w with P's two bits as constants,
     * updating masks ul/uh (undecided) and pl/ph (perturbed) with suffix sfx */
    void emit_level(const char* ind, uint32_t w, uint32_t h, const std::string& sfx, const char* ps) {
        const uint32_t b0 = (Pv >> (31 - 2 * h)) & 1u;
        const uint32_t b1 = (Pv >> (30 - 2 * h)) & 1u;
        const char* S = sfx.c_str();
        o << ind << fmt("{ const uint4 x = pbn_philox_draw(P, %s, %s);", ps, hex32((PBN_DOM_PERT << 28) | (w << 4) | h).c_str());
        if (b0) o << fmt(" pl%s |= ul%s & ~x.x; ph%s |= uh%s & ~x.y; ul%s &= x.x; uh%s &= x.y;", S, S, S, S, S, S);
        else o << fmt(" ul%s &= ~x.x; uh%s &= ~x.y;", S, S);
        if (b1) o << fmt(" pl%s |= ul%s & ~x.z; ph%s |= uh%s & ~x.w; ul%s &= x.z; uh%s &= x.w;", S, S, S, S, S, S);
        else o << fmt(" ul%s &= ~x.z; uh%s &= ~x.w;", S, S);
        o << " }\n";
    }

    /* the rolled loop over the remaining level pairs h0.. of words w (and w + 1) */
    void emit_level_loop(uint32_t w, bool two, uint32_t h0, const std::string& s0, const std::string& s1, const char* ps) {
        o << "        { uint32_t pp = " << hex32(h0 ? (Pv << (2 * h0)) : Pv) << ";\n"
          << "#pragma unroll 1\n"
          << "        for (uint32_t h = " << h0 << "u; h < " << hmax << "u; ++h) {\n"
          << "          if (!(ul" << s0 << " | uh" << s0 << (two ? " | ul" + s1 + " | uh" + s1 : std::string()) << ")) break;\n"
          << "          const uint32_t m0 = (uint32_t)((int32_t)pp >> 31), m1 = (uint32_t)((int32_t)(pp << 1) >> 31);\n"
          << "          pp <<= 2;\n"
          << "          const uint4 x0 = pbn_philox_draw(P, " << ps << ", " << hex32((PBN_DOM_PERT << 28) | (w << 4)) << " | h);\n";
        if (two)
            o << "          const uint4 x1 = pbn_philox_draw(P, " << ps << ", " << hex32((PBN_DOM_PERT << 28) | ((w + 1) << 4))
              << " | h);\n";
        for (int k = 0; k < (two ? 2 : 1); ++k) {
            const char* S = (k ? s1 : s0).c_str();
            o << fmt("          pl%s |= ul%s & ~x%d.x & m0; ph%s |= uh%s & ~x%d.y & m0; ul%s &= ~(x%d.x ^ m0); uh%s &= ~(x%d.y ^ m0);\n",
                     S, S, k, S, S, k, S, k, S, k)
              << fmt("          pl%s |= ul%s & ~x%d.z & m1; ph%s |= uh%s & ~x%d.w & m1; ul%s &= ~(x%d.z ^ m1); uh%s &= ~(x%d.w ^ m1);\n",
                     S, S, k, S, S, k, S, k, S, k);
        }
        o << "        } }\n";
    }

    /* choice of a multi-function node from its SEL slot's thresholds */
    std::string choice_expr(const pbn_img_multi& M) const {
        if (ws_choices_ || ch_smem_) {
            const uint32_t* ss = selslot + 4 * ((M.ch_off & 3u) * H.n_sel + (M.ch_off >> 2));
            if (!ss[2]) return std::string();
            /* warp split: the choice computed right after its block's draw, or read from
             * the choice bytes the warps wrote in phase A */
            return ch_smem_ ? fmt("((uint32_t)CHs[%uu])", 32u * M.ch_off) : fmt("J%u", M.ch_off);
        }
        return slot_choice(M.ch_off);
    }

    /* choice of the node in SEL slot `slot` from its block's uniforms U<slot/4> */
    std::string slot_choice(uint32_t slot) const {
        const std::string u = fmt("U%u.%c", slot / 4, lanes[slot % 4]);
        const uint32_t* ss = selslot + 4 * ((slot & 3u) * H.n_sel + (slot >> 2)); /* t1, t2, n_thr, first */
        const uint32_t n_thr = ss[2];
        std::string j;
        for (uint32_t q = 0; q < n_thr; ++q) {
            const uint32_t T = n_thr <= 2 ? ss[q] : thr[ss[3] + q];
            j += (q ? " + " : "") + fmt("(uint32_t)(%s >= %s)", u.c_str(), hex32(T).c_str());
        }
        return j;
    }

    /* input pattern of k inputs from chunked records `stride` chunks apart (32 in
     * the row-interleaved group layout, 1 for a split node's functions) */
    std::string pattern(uint32_t in_chunk, uint32_t k, uint32_t stride) const {
        std::string xexpr;
        for (uint32_t b = 0; b < k; ++b) {
            const uint32_t rec = inrec[4 * (in_chunk + stride * (b / 4)) + (b & 3)];
            const uint32_t row = rec >> 7, bit = ((b & 3) + (rec & 31)) & 31;
            xexpr += (b ? " | " : "") + gather(row, bit, b);
        }
        return xexpr.empty() ? std::string("0u") : xexpr;
    }

    std::vector<uint32_t> blocks_of(uint32_t gi) const {
        std::vector<uint32_t> b;
        const pbn_img_group& G = groups[gi];
        for (uint32_t m = 0; m < G.n_mul; ++m) b.push_back(multi[G.mul_first + 32 * m].ch_off / 4);
        return b;
    }

    /* split node: every function's pattern is a few register operations; the selected
     * one's table bit is kept (immediates when every table fits in 64 bits, else one
     * lookup at the selected table) */
    void emit_split_group(uint32_t r, const pbn_img_group& G) {
        std::string j = choice_expr(multi[G.mul_first]);
        if (j.empty()) j = "0u";
        o << "const uint32_t j = " << j << "; ";
        bool small = true;
        for (uint32_t f = 0; f < G.q; ++f) small = small && (subs[2 * (G.tab_off + 32 * f)] >> 27) <= 6;
        std::string v = "0u";
        if (small) {
            for (uint32_t f = G.q; f-- > 0;) {
                const uint32_t* F = subs + 2 * (G.tab_off + 32 * f);
                const uint32_t k = F[0] >> 27, ch = F[0] & 0x7FFFFFFu;
                const uint64_t t64 = (k == 6 ? ((uint64_t)tab[F[1] + 1] << 32) : 0ull) | tab[F[1]];
                const std::string vf =
                    fmt("(uint32_t)((0x%016llxull >> (", (unsigned long long)t64) + pattern(ch, k, 1) + ")) & 1ull)";
                v = f + 1 == G.q ? vf : fmt("(j == %uu ? ", f) + vf + " : " + v + ")";
            }
        } else {
            std::string xs = "0u", offs = "0u";
            for (uint32_t f = G.q; f-- > 0;) {
                const uint32_t* F = subs + 2 * (G.tab_off + 32 * f);
                const std::string xf = "(" + pattern(F[0] & 0x7FFFFFFu, F[0] >> 27, 1) + ")";
                xs = f + 1 == G.q ? xf : fmt("(j == %uu ? ", f) + xf + " : " + xs + ")";
                offs = f + 1 == G.q ? fmt("%uu", F[1]) : fmt("(j == %uu ? %uu : ", f, F[1]) + offs + ")";
            }
            o << "const uint32_t x = " << xs << "; const uint32_t to = " << offs << "; ";
            v = tab_smem ? "((TAB[to + (x >> 5)] >> (x & 31u)) & 1u)"
                         : "((__ldg(TAB + to + (x >> 5)) >> (x & 31u)) & 1u)";
        }
        o << "n" << r << " |= " << v << " << " << (uint32_t)G.shift << "; }\n";
    }

    /* merged group: combined choice, input pattern (single-bit or multiply gathers)
     * and the table entry (an immediate for tables of at most 64 bits) */
    void emit_merged_group(uint32_t r, uint32_t gi, const pbn_img_group& G) {
        std::string cexpr;
        for (uint32_t m = 0; m < G.n_mul; ++m) {
            const pbn_img_multi& M = multi[G.mul_first + 32 * m];
            const std::string j = choice_expr(M);
            if (j.empty()) continue;
            cexpr += (cexpr.empty() ? "" : " + ") + (M.radix == 1 ? "(" + j + ")" : fmt("%uu * (", M.radix) + j + ")");
        }
        const GPlan& GP = gp[gi];
        const uint32_t q = GP.used ? GP.qn : G.q;
        if (GP.used) {
            std::string xe;
            for (const GTerm& t : GP.terms) {
                std::string term;
                if (t.magic) {
                    const MagicTerm& m = t.m;
                    term = fmt("((((s%u & %s) * %s) >> %u) & %s)", m.row, hex32(m.mask).c_str(), hex32(m.mul).c_str(),
                               m.shift, hex32((1u << m.width) - 1u).c_str());
                    if (t.off) term = "(" + term + fmt(" << %u)", t.off);
                } else {
                    term = gather(t.row, t.bit, t.off);
                }
                xe += (xe.empty() ? "" : " | ") + term;
            }
            o << "const uint32_t x = " << xe << "; ";
        } else {
            o << "const uint32_t x = " << pattern(G.in_chunk, q, 32) << "; ";
        }
        if (!cexpr.empty()) o << "const uint32_t e = ((" << cexpr << ") << " << q << ") | x; ";
        else o << "const uint32_t e = x; ";
        const uint32_t l2w = G.l2w;
        const uint32_t ebits = 1u << l2w;
        const uint32_t emask = ebits >= 32 ? 0xFFFFFFFFu : ((1u << ebits) - 1u);
        /* size of this group's table in words: up to the next table's offset, or the end */
        auto nx = std::upper_bound(tab_starts.begin(), tab_starts.end(), G.tab_off);
        const uint32_t toff = GP.used ? GP.tab_off : G.tab_off;
        const uint32_t tab_words = GP.used ? GP.tab_words
                                           : (nx == tab_starts.end() ? (H.off_ret - H.off_tables) / 4 : *nx) - G.tab_off;
        const uint32_t* tabv = magic ? tabm.data() : tab;
        std::string v;
        if (tab_words == 1) {
            v = fmt("((%s >> (e << %u)) & %s)", hex32(tabv[toff]).c_str(), l2w, hex32(emask).c_str());
        } else if (tab_words == 2) {
            const uint64_t t64 = ((uint64_t)tabv[toff + 1] << 32) | tabv[toff];
            v = fmt("((uint32_t)(0x%016llxull >> (e << %u)) & %s)", (unsigned long long)t64, l2w, hex32(emask).c_str());
        } else if (tab_smem) {
            v = fmt("((TAB[%uu + ((e << %u) >> 5)] >> ((e << %u) & 31u)) & %s)", toff, l2w, l2w, hex32(emask).c_str());
        } else {
            v = fmt("((__ldg(TAB + %uu + ((e << %u) >> 5)) >> ((e << %u) & 31u)) & %s)", toff, l2w, l2w,
                    hex32(emask).c_str());
        }
        o << "n" << r << " |= " << v << " << " << (uint32_t)G.shift << "; }\n";
    }

    /* merged-table evaluation of every group from s and the SEL uniforms U: n<row>.
     * Wide plans take the groups in the order of the last SEL block they read and
     * draw each block just before its first use. */
    void emit_eval() {
        for (uint32_t r = 0; r < H.W32; ++r) o << "        uint32_t n" << r << " = 0;\n";
        const uint32_t* wgroups = V.at<uint32_t>(H.off_wgroups);
        std::vector<std::pair<uint32_t, uint32_t>> order; /* (row, group) */
        for (uint32_t r = 0; r < H.W32; ++r)
            for (uint32_t i = words[r].x; i < words[r].x + words[r].y; ++i) order.push_back({r, wgroups[i]});
        std::vector<uint8_t> drawn(H.n_sel, 0);
        if (wide) {
            std::stable_sort(order.begin(), order.end(), [&](const std::pair<uint32_t, uint32_t>& x,
                                                             const std::pair<uint32_t, uint32_t>& y) {
                const auto bx = blocks_of(x.second), by = blocks_of(y.second);
                const uint32_t mx = bx.empty() ? 0 : *std::max_element(bx.begin(), bx.end());
                const uint32_t my = by.empty() ? 0 : *std::max_element(by.begin(), by.end());
                return mx < my;
            });
        }
        for (const auto& ri : order) {
            const uint32_t r = ri.first;
            const uint32_t gi = ri.second;
            const pbn_img_group& G = groups[gi];
            if (wide)
                for (uint32_t b : blocks_of(gi))
                    if (!drawn[b]) {
                        drawn[b] = 1;
                        o << "        const uint4 U" << b << " = pbn_philox_draw(P, ps, "
                          << hex32((PBN_DOM_SEL << 28) | selblk[b]) << ");\n";
                    }
            o << "        { ";
            if (G.l2w == PBN_IMG_SPLIT) emit_split_group(r, G);
            else emit_merged_group(r, gi, G);
        }
    }

    /* meta-state counts and the optional trace of the new state */
    void emit_counts() {
        o << "      { const uint32_t z = " << z << ";\n"
             "        const uint32_t cv = k >= P.kv0 ? 1u : 0u, cp = k >= P.kp0 ? 1u : 0u;\n"
             "        cV += cv & z; c11 += cp & zp & z; c01 += cp & (zp ^ 1u) & z; c10 += cp & zp & (z ^ 1u); zp = z; }\n";
        o << "      if (P.trace && (k + 1) % P.trace_stride == 0) {\n"
             "        const uint64_t snap = (k + 1) / P.trace_stride - 1;\n";
        for (uint32_t r = 0; r < H.W32; r += 2)
            o << "        P.trace[(snap * " << H.W32 / 2 << "u + " << r / 2 << "u) * P.n_traj + lt] = ((uint64_t)s"
              << r + 1 << " << 32) | s" << r << ";\n";
        o << "      }\n";
    }

    /* Software-pipelined steps: every random draw is independent of the state, so
     * the SEL blocks and the first perturbation level pairs of step t + 1 are drawn
     * while step t's groups are evaluated (one block of independent work); the
     * evaluation always runs and a select keeps s XOR flips in perturbed steps. */
    void emit_pipelined_steps() {
        const uint32_t npeel = std::min<uint32_t>(hmax, 3u);
        o << "    pbn_philox_step ps = pbn_philox_begin(P, traj, P.step_begin);\n";
        emit_sel_draws("    ", "uint4 ", "U", "ps");
        for (uint32_t w = 0; w < H.W; ++w) {
            const uint64_t v = Pv ? valid_of(w) : 0ull;
            o << fmt("    uint32_t ul%u = %s, uh%u = %s, pl%u = 0, ph%u = 0;\n", w, hex32((uint32_t)v).c_str(), w,
                     hex32((uint32_t)(v >> 32)).c_str(), w, w);
            for (uint32_t h = 0; h < npeel; ++h) emit_level("    ", w, h, std::to_string(w), "ps");
        }
        o << "    for (uint32_t k = 0; k < P.n_steps; ++k) {\n"
             "      const uint64_t t = P.step_begin + k;\n"
             "      uint32_t any = 0;\n      uint32_t";
        for (uint32_t r = 0; r < H.W32; ++r) o << (r ? ", " : " ") << "f" << r << " = 0";
        o << ";\n";
        /* the remaining level pairs of step t, then its flips */
        if (Pv && hmax > npeel)
            for (uint32_t w = 0; w < H.W; w += 2)
                emit_level_loop(w, w + 1 < H.W, npeel, std::to_string(w), std::to_string(w + 1), "ps");
        for (uint32_t w = 0; w < H.W && Pv; ++w) {
            o << "      if (pl" << w << " | ph" << w << ") {\n          any = 1u;\n";
            emit_flips(w, "pl" + std::to_string(w), "ph" + std::to_string(w), "f", "|=");
            o << "      }\n";
        }
        /* draws of step t + 1 */
        o << "      const pbn_philox_step psn = pbn_philox_begin(P, traj, t + 1);\n";
        emit_sel_draws("      ", "const uint4 ", "V", "psn");
        for (uint32_t w = 0; w < H.W && Pv; ++w) {
            const uint64_t v = valid_of(w);
            const std::string S = "n" + std::to_string(w);
            o << fmt("      uint32_t ul%s = %s, uh%s = %s, pl%s = 0, ph%s = 0;\n", S.c_str(), hex32((uint32_t)v).c_str(),
                     S.c_str(), hex32((uint32_t)(v >> 32)).c_str(), S.c_str(), S.c_str());
            for (uint32_t h = 0; h < npeel; ++h) emit_level("      ", w, h, S, "psn");
        }
        /* evaluation of step t and the new state */
        o << "      {\n";
        emit_eval();
        for (uint32_t r = 0; r < H.W32; ++r) {
            if (nodewise) o << "        s" << r << " = (n" << r << " & ~f" << r << ") | (~s" << r << " & f" << r << ");\n";
            else o << "        s" << r << " = any ? (s" << r << " ^ f" << r << ") : n" << r << ";\n";
        }
        o << "      }\n";
        emit_counts();
        /* rotate */
        o << "      ps = psn;\n";
        for (uint32_t i = 0; i < H.n_sel; ++i) o << "      U" << i << " = V" << i << ";\n";
        for (uint32_t w = 0; w < H.W && Pv; ++w)
            o << fmt("      ul%u = uln%u; uh%u = uhn%u; pl%u = pln%u; ph%u = phn%u;\n", w, w, w, w, w, w, w, w);
        o << "    }\n";
    }

    /* geometric sampler: per word pair one block; the common case is one 64-bit
     * compare per word against G[L-1]; otherwise the perturbed lanes are found one by
     * one */
    void emit_geometric_perturbation(const char* ftarget, const char* fop) {
        const uint64_t* G = V.at<uint64_t>(H.off_geo);
        for (uint32_t wp = 0; 2 * wp < H.W; ++wp) {
            if (!pair_selected(wp)) continue;
            o << "      { const uint4 g0 = pbn_philox_draw(P, ps, " << hex32((PBN_DOM_GEO << 28) | (wp << 8)) << ");\n";
            for (uint32_t h2 = 0; h2 < 2 && 2 * wp + h2 < H.W; ++h2) {
                const uint32_t w = 2 * wp + h2;
                const uint32_t L = (w == H.W - 1 && (H.n & 63u)) ? (H.n & 63u) : 64u;
                const char* lo = h2 ? "z" : "x";
                const char* hi = h2 ? "w" : "y";
                o << fmt("        { uint64_t U = ((uint64_t)g0.%s << 32) | g0.%s;\n", hi, lo)
                  << fmt("          if (U < 0x%016llxull) {\n", (unsigned long long)G[L - 1])
                  << "            uint32_t pl = 0, ph = 0, pos = 0, j = 0;\n"
                  << "            for (;;) {\n"
                  << fmt("              if (U >= GEO_T%s[%uu - pos - 1]) break;\n", sfx_.c_str(), L)
                  << "              uint32_t k = 0;\n              while (U >= GEO_T" << sfx_ << "[k]) ++k;\n"
                  << "              const uint32_t b = pos + k;\n"
                  << "              if (b < 32) pl |= 1u << b; else ph |= 1u << (b - 32);\n"
                  << fmt("              pos = b + 1;\n              if (pos >= %uu) break;\n", L)
                  << "              ++j;\n"
                  << "              const uint4 x = pbn_philox_draw(P, ps, " << hex32((PBN_DOM_GEO << 28) | (wp << 8)) << " | j);\n"
                  << fmt("              U = ((uint64_t)x.%s << 32) | x.%s;\n", hi, lo)
                  << "            }\n            any = 1u;\n";
                emit_flips(w, "pl", "ph", ftarget, fop);
                o << "          }\n        }\n";
            }
            o << "      }\n";
        }
    }

    /* one word at a time, every level pair unrolled with its P bits as constants */
    void emit_unrolled_perturbation(const char* ftarget, const char* fop) {
        for (uint32_t w = 0; w < H.W; ++w) {
            if (!pair_selected(w / 2)) continue;
            const uint64_t valid = valid_of(w);
            o << "      { uint32_t ul = " << hex32((uint32_t)valid) << ", uh = " << hex32((uint32_t)(valid >> 32))
              << ", pl = 0, ph = 0;\n";
            for (uint32_t h = 0; h < hmax; ++h) {
                o << "        if (ul | uh) ";
                emit_level("", w, h, "", "ps");
            }
            o << "        if (pl | ph) {\n          any = 1u;\n";
            emit_flips(w, "pl", "ph", ftarget, fop);
            o << "        }\n      }\n";
        }
    }

    /* words in pairs: one rolled loop draws both words' level pairs, two independent
     * Philox chains per iteration; interleaved: the first level pairs (needed by a
     * 64-lane word with probability ~1) are straight-line */
    void emit_paired_perturbation(const char* ftarget, const char* fop) {
        const uint32_t npeel = interleave ? std::min<uint32_t>(hmax, 3u) : 0u;
        for (uint32_t w = 0; w < H.W; w += 2) {
            if (!pair_selected(w / 2)) continue;
            const bool two = w + 1 < H.W;
            const uint64_t v0 = valid_of(w), v1 = two ? valid_of(w + 1) : 0ull;
            o << "      { uint32_t ul0 = " << hex32((uint32_t)v0) << ", uh0 = " << hex32((uint32_t)(v0 >> 32))
              << ", pl0 = 0, ph0 = 0";
            if (two) o << ", ul1 = " << hex32((uint32_t)v1) << ", uh1 = " << hex32((uint32_t)(v1 >> 32)) << ", pl1 = 0, ph1 = 0";
            o << ";\n";
            for (uint32_t h = 0; h < npeel; ++h)
                for (uint32_t k2 = 0; k2 < (two ? 2u : 1u); ++k2) emit_level("        ", w + k2, h, std::to_string(k2), "ps");
            emit_level_loop(w, two, npeel, "0", "1", "ps");
            o << "        if (pl0 | ph0) {\n          any = 1u;\n";
            emit_flips(w, "pl0", "ph0", ftarget, fop);
            o << "        }\n";
            if (two) {
                o << "        if (pl1 | ph1) {\n          any = 1u;\n";
                emit_flips(w + 1, "pl1", "ph1", ftarget, fop);
                o << "        }\n";
            }
            o << "      }\n";
        }
    }

    /* the step loop: perturbation (P's levels compiled in), then, in a non-perturbed
     * step (every step with node-wise semantics), selection and evaluation; counts */
    void emit_steps() {
        o << "    for (uint32_t k = 0; k < P.n_steps; ++k) {\n"
             "      const uint64_t t = P.step_begin + k;\n"
             "      const pbn_philox_step ps = pbn_philox_begin(P, traj, t);\n"
             "      uint32_t any = 0;\n";
        if (nodewise) {
            o << "      uint32_t";
            for (uint32_t r = 0; r < H.W32; ++r) o << (r ? ", " : " ") << "g" << r << " = 0";
            o << ";\n";
        }
        const char* ftarget = nodewise ? "g" : "s";
        const char* fop = nodewise ? "|=" : "^=";
        /* interleaved: the SEL blocks are drawn before the perturbation check (they are
         * needed in every non-perturbed step), so that their Philox chains and the first
         * perturbation levels form one block of independent work */
        if (interleave) emit_sel_draws("      ", "const uint4 ", "U", "ps");
        if (Pv && geometric) emit_geometric_perturbation(ftarget, fop);
        else if (Pv && (flags_ & PBN_COMPILE_PERT_UNROLLED)) emit_unrolled_perturbation(ftarget, fop);
        else if (Pv) emit_paired_perturbation(ftarget, fop);
        o << (nodewise ? "      {\n" : "      if (!any) {\n");
        if (!interleave && !wide) emit_sel_draws("        ", "const uint4 ", "U", "ps");
        emit_eval();
        for (uint32_t r = 0; r < H.W32; ++r) {
            if (nodewise) o << "        s" << r << " = (n" << r << " & ~g" << r << ") | (~s" << r << " & g" << r << ");\n";
            else o << "        s" << r << " = n" << r << ";\n";
        }
        o << "      }\n";
        emit_counts();
        o << "    }\n";
    }

    /* the state and counts written back, pooled counts reduced per warp */
    void emit_epilogue() {
        if (bs_) {
            for (uint32_t r = 0; r < H.W32; r += 2)
                o << "    P.state[(uint64_t)" << r / 2 << " * P.n_traj + lt] = ((uint64_t)s" << r + 1 << " << 32) | s" << r
                  << ";\n";
            o << "    if (P.counts) {\n"
                 "      const uint64_t nt = P.n_traj;\n"
                 "      P.counts[lt] += cV; P.counts[nt + lt] += P.pairs - c01 - c10 - c11;\n"
                 "      P.counts[2 * nt + lt] += c01; P.counts[3 * nt + lt] += c10; P.counts[4 * nt + lt] += c11;\n"
                 "    }\n  }\n";
            o << "  cnt[0] = cV; cnt[1] = c01; cnt[2] = c10; cnt[3] = c11;\n  return active;\n}\n";
            return;
        }
        for (uint32_t r = 0; r < H.W32; r += 2)
            o << "    P.state[(uint64_t)" << r / 2 << " * P.n_traj + lt] = ((uint64_t)s" << r + 1 << " << 32) | s" << r << ";\n";
        o << "    if (P.counts) {\n"
             "      const uint64_t nt = P.n_traj;\n"
             "      P.counts[lt] += cV; P.counts[nt + lt] += P.pairs - c01 - c10 - c11;\n"
             "      P.counts[2 * nt + lt] += c01; P.counts[3 * nt + lt] += c10; P.counts[4 * nt + lt] += c11;\n"
             "    }\n  }\n";
        o << "  if (P.pooled) {\n"
             "    uint64_t v[5] = {active ? cV : 0u, active ? (uint64_t)(P.pairs - c01 - c10 - c11) : 0u,\n"
             "                     active ? c01 : 0u, active ? c10 : 0u, active ? c11 : 0u};\n"
             "#pragma unroll\n    for (int i = 0; i < 5; ++i) {\n"
             "#pragma unroll\n      for (int d = 16; d > 0; d >>= 1) v[i] += __shfl_xor_sync(0xFFFFFFFFu, v[i], d);\n    }\n"
             "    if ((threadIdx.x & 31u) == 0) {\n"
             "      for (int i = 0; i < 5; ++i) if (v[i]) atomicAdd(P.pooled + i, (unsigned long long)v[i]);\n    }\n  }\n";
        o << "}\n";
    }
};

bool generate(const pbn_plan& plan, uint32_t flags, Generated* out, std::string* why) {
    KernelSource ks(plan, flags);
    return ks.generate(out, why);
}

const char kBatchHeader[] =
#include "pbn_batch_cuh.inc"
    ;

/* ---- nvJitLink, loaded on first use ----------------------------------------------------- */
typedef struct _nvJitLinkHandle* nvJitLinkHandle_t;
struct JitLink {
    int (*create)(nvJitLinkHandle_t*, uint32_t, const char**);
    int (*destroy)(nvJitLinkHandle_t*);
    int (*add_data)(nvJitLinkHandle_t, int, const void*, size_t, const char*);
    int (*complete)(nvJitLinkHandle_t);
    int (*cubin_size)(nvJitLinkHandle_t, size_t*);
    int (*cubin)(nvJitLinkHandle_t, void*);
    int (*log_size)(nvJitLinkHandle_t, size_t*);
    int (*log)(nvJitLinkHandle_t, char*);
    bool ok = false;
    std::string err;
};

JitLink& jitlink() {
    static JitLink N;
    static std::once_flag once;
    std::call_once(once, [] {
        const char* names[] = {"libnvJitLink.so.13", "libnvJitLink.so", "/usr/local/cuda/lib64/libnvJitLink.so.13",
                               "/usr/local/cuda/lib64/libnvJitLink.so"};
        void* h = nullptr;
        for (const char* nm : names)
            if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
        if (!h) {
            N.err = "libnvJitLink not found";
            return;
        }
        /* the library exports versioned names (the header maps the plain ones to them) */
        auto sym = [&](const char* base) -> void* {
            void* p = dlsym(h, (std::string("__") + base + "_13_0").c_str());
            return p ? p : dlsym(h, base);
        };
#define PBN_LSYM(field, name)                                     \
    *reinterpret_cast<void**>(&N.field) = sym(name);              \
    if (!N.field) {                                               \
        N.err = std::string("libnvJitLink lacks ") + name;        \
        return;                                                   \
    }
        PBN_LSYM(create, "nvJitLinkCreate");
        PBN_LSYM(destroy, "nvJitLinkDestroy");
        PBN_LSYM(add_data, "nvJitLinkAddData");
        PBN_LSYM(complete, "nvJitLinkComplete");
        PBN_LSYM(cubin_size, "nvJitLinkGetLinkedCubinSize");
        PBN_LSYM(cubin, "nvJitLinkGetLinkedCubin");
        PBN_LSYM(log_size, "nvJitLinkGetErrorLogSize");
        PBN_LSYM(log, "nvJitLinkGetErrorLog");
#undef PBN_LSYM
        N.ok = true;
    });
    return N;
}

/* The interpreter's relocatable work-item function, built with the library into the
 * same directory (pbn_batch_item.cubin). */
bool read_item_cubin(std::vector<char>* out, std::string* why) {
    Dl_info di;
    if (!dladdr(reinterpret_cast<void*>(&read_item_cubin), &di) || !di.dli_fname) {
        *why = "cannot locate the library's directory";
        return false;
    }
    std::string path(di.dli_fname);
    const size_t cut = path.find_last_of('/');
    path = (cut == std::string::npos ? std::string(".") : path.substr(0, cut)) + "/pbn_batch_item.cubin";
    FILE* f = fopen(path.c_str(), "rb");
    if (!f) {
        *why = "missing " + path;
        return false;
    }
    fseek(f, 0, SEEK_END);
    const long sz = ftell(f);
    fseek(f, 0, SEEK_SET);
    out->resize(sz > 0 ? (size_t)sz : 0);
    const bool ok = sz > 0 && fread(out->data(), 1, (size_t)sz, f) == (size_t)sz;
    fclose(f);
    if (!ok) *why = "cannot read " + path;
    return ok;
}

}  // namespace

namespace pbn {

bool jit_batch_function(const pbn_plan* plan, uint32_t flags, const JitBatchNet& spec, std::string* src,
                        uint32_t* tab_bytes, std::string* why) {
    KernelSource ks(*plan, flags, &spec);
    Generated gen;
    if (!ks.generate(&gen, why)) return false;
    *src = std::move(gen.src);
    *tab_bytes = gen.tab_bytes;
    return true;
}

namespace {
/* NVRTC compile of one program of the batch module (relocatable when `rdc`). */
bool nvrtc_cubin(const std::string& src, const char* name, bool rdc, std::vector<char>* cubin, std::string* log) {
    Nvrtc& N = nvrtc();
    nvrtcProgram_t prog = nullptr;
    const char* hdrs[] = {kDeviceHeader, kBatchHeader};
    const char* hnames[] = {"pbn_device.cuh", "pbn_batch.cuh"};
    if (N.create(&prog, src.c_str(), name, 2, hdrs, hnames) != 0) {
        *log = "nvrtcCreateProgram failed";
        return false;
    }
    std::vector<const char*> opts = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo", "--maxrregcount=128"};
    if (rdc) opts.push_back("--relocatable-device-code=true");
    const int rc = N.compile(prog, (int)opts.size(), opts.data());
    size_t ls = 0;
    N.log_size(prog, &ls);
    std::string clog(ls, '\0');
    if (ls) N.log(prog, &clog[0]);
    if (rc != 0) {
        N.destroy(&prog);
        *log = clog;
        return false;
    }
    size_t cs = 0;
    N.cubin_size(prog, &cs);
    cubin->resize(cs);
    N.cubin(prog, cubin->data());
    N.destroy(&prog);
    return true;
}
}  // namespace

int jit_batch_module(const std::vector<std::string>& functions, const std::vector<uint32_t>& compiled, bool interp,
                     uint32_t threads, void** library, void** kernel, double* ms, std::string* log) {
    auto t0 = std::chrono::steady_clock::now();
    Nvrtc& N = nvrtc();
    if (!N.ok) {
        *log = N.err;
        return fail(PBN_ECUDA, "NVRTC unavailable: %s", N.err.c_str());
    }
    /* the dispatching persistent kernel */
    std::ostringstream o;
    o << "#include \"pbn_batch.cuh\"\n";
    for (uint32_t i : compiled)
        o << "extern \"C\" __device__ bool pbn_net_" << i
          << "(const pbn_netdesc& D, const pbn_workitem W, const uint64_t step_offset, const uint32_t n_steps, "
             "uint32_t* cnt, const uint8_t* kernel_smem, uint32_t* status);\n";
    if (interp)
        o << "extern \"C\" __device__ bool pbn_batch_interp_item(uint64_t step_offset, uint32_t n_steps, "
             "const pbn_workitem* W, const pbn_netdesc* D, const uint32_t* meta_sh, uint32_t* c, "
             "const uint8_t* kernel_smem, uint32_t* status);\n";
    o << "extern \"C\" __global__ void __launch_bounds__(" << threads << ", 1) pbn_cbatch_kernel(const pbn_batch_params B) {\n"
         "  extern __shared__ __align__(128) uint8_t smem[];\n"
         "  __shared__ __align__(8) uint64_t bar;\n  __shared__ uint32_t item_sh;\n"
         "  __shared__ uint32_t meta_sh[3 * PBN_BATCH_META_ROWS];\n"
         "  pbn_batch_loop(B, smem, &bar, &item_sh, meta_sh,\n"
         "    [&](const pbn_workitem& W, const pbn_netdesc& D, const uint32_t* ms, uint32_t c[4]) -> bool {\n"
         "      switch (W.net) {\n";
    for (uint32_t i : compiled)
        o << "        case " << i << "u: return pbn_net_" << i << "(D, W, B.step_offset, B.n_steps, c, smem, B.status);\n";
    if (interp)
        o << "        default: return pbn_batch_interp_item(B.step_offset, B.n_steps, &W, &D, ms, c, smem, B.status);\n";
    else o << "        default: return false;\n";
    o << "      }\n    });\n}\n";
    /* the network functions in up to `parts` programs compiled in parallel (each a
     * relocatable unit), then linked with the dispatcher (and the interpreter) */
    unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    if (const char* t = getenv("PBN_BATCH_COMPILE_THREADS")) hw = std::max(1, atoi(t));
    const size_t parts = std::min<size_t>(functions.size(), std::min<unsigned>(hw, 32u));
    std::vector<std::string> srcs(parts + 1);
    srcs[0] = o.str();
    for (size_t k = 0; k < functions.size(); ++k) {
        std::string& dst = srcs[1 + k * parts / functions.size()];
        if (dst.empty()) dst = "#include \"pbn_batch.cuh\"\n";
        dst += functions[k];
    }
    /* PBN_BATCH_MODULE_DUMP=<path>: write the generated sources there (inspection) */
    if (const char* dump = getenv("PBN_BATCH_MODULE_DUMP")) {
        if (FILE* f = fopen(dump, "w")) {
            for (const std::string& x : srcs) fwrite(x.data(), 1, x.size(), f);
            fclose(f);
        }
    }
    std::vector<std::vector<char>> cubins(srcs.size());
    std::vector<std::string> logs(srcs.size());
    std::vector<char> okv(srcs.size(), 0);
    {
        std::vector<std::thread> th;
        for (size_t k = 0; k < srcs.size(); ++k)
            th.emplace_back([&, k] {
                const std::string nm = "pbn_batch_module_" + std::to_string(k) + ".cu";
                okv[k] = nvrtc_cubin(srcs[k], nm.c_str(), true, &cubins[k], &logs[k]) ? 1 : 0;
            });
        for (auto& t : th) t.join();
    }
    for (size_t k = 0; k < srcs.size(); ++k)
        if (!okv[k]) {
            *log = logs[k];
            return fail(PBN_ECUDA, "NVRTC compilation of the batch module failed: %.400s", logs[k].c_str());
        }
    std::vector<char> item;
    if (interp) {
        std::string why;
        if (!read_item_cubin(&item, &why)) {
            *log = why;
            return fail(PBN_ECUDA, "batch module: %s", why.c_str());
        }
    }
    JitLink& L = jitlink();
    if (!L.ok) {
        *log = L.err;
        return fail(PBN_ECUDA, "nvJitLink unavailable: %s", L.err.c_str());
    }
    nvJitLinkHandle_t h = nullptr;
    const char* lopts[] = {"-arch=sm_103a"};
    int lr = L.create(&h, 1, lopts);
    const int kCubin = 1; /* NVJITLINK_INPUT_CUBIN */
    for (size_t k = 0; k < cubins.size() && lr == 0; ++k)
        lr = L.add_data(h, kCubin, cubins[k].data(), cubins[k].size(), "pbn_batch_module");
    if (lr == 0 && interp) lr = L.add_data(h, kCubin, item.data(), item.size(), "pbn_batch_item");
    if (lr == 0) lr = L.complete(h);
    if (lr != 0) {
        size_t n = 0;
        if (h) L.log_size(h, &n);
        std::string el(n, '\0');
        if (n) L.log(h, &el[0]);
        if (h) L.destroy(&h);
        *log = el;
        return fail(PBN_ECUDA, "nvJitLink failed (%d): %.400s", lr, el.c_str());
    }
    size_t n = 0;
    L.cubin_size(h, &n);
    std::vector<char> linked(n);
    L.cubin(h, linked.data());
    L.destroy(&h);
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, linked.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&kern, lib, "pbn_cbatch_kernel");
    if (e != cudaSuccess) {
        if (lib) cudaLibraryUnload(lib);
        *log = cudaGetErrorString(e);
        return fail(PBN_ECUDA, "loading the batch module failed: %s", cudaGetErrorString(e));
    }
    *library = lib;
    *kernel = reinterpret_cast<void*>(kern);
    if (ms) *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return PBN_OK;
}

void jit_library_unload(void* library) {
    if (library) cudaLibraryUnload(static_cast<cudaLibrary_t>(library));
}

}  // namespace pbn

/* ---- compiled-plan cache and launch (called from pbn_sim.cu and the C ABI) --------- */
struct pbn_jit_state {
    std::mutex mu;
    int state = 0;  /* 0: not tried, 1: compiled, -1: failed */
    uint32_t flags = 0;
    std::string log;
    std::string src;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    uint32_t tab_bytes = 0;
    uint32_t warps = 0;  /* warp-split form: warps per CTA of 32 trajectories */
    uint32_t dyn_smem = 0; /* dynamic shared memory of a launch (0: tab_bytes) */
    uint32_t static_smem = 1024; /* upper bound of the kernel's static shared memory */
    double compile_ms = 0;
};

namespace pbn {

pbn_jit_state* jit_state(const pbn_plan* plan) {
    static std::mutex g;
    std::lock_guard<std::mutex> lk(g);
    if (!plan->jit) plan->jit = new pbn_jit_state();
    return plan->jit;
}

void jit_free(pbn_jit_state* J) {
    if (!J) return;
    if (J->lib) cudaLibraryUnload(J->lib);
    delete J;
}

int jit_compile(const pbn_plan* plan, uint32_t flags) {
    pbn_jit_state* J = jit_state(plan);
    std::lock_guard<std::mutex> g(J->mu);
    if (J->state == 1 && J->flags == flags) return PBN_OK;
    if (J->state == -1 && J->flags == flags) return fail(PBN_EINVAL, "plan compilation failed earlier: %s", J->log.c_str());
    if (J->lib) {
        cudaLibraryUnload(J->lib);
        J->lib = nullptr;
        J->kern = nullptr;
    }
    J->state = 0;
    J->flags = flags;
    Generated gen;
    std::string why;
    if (!generate(*plan, flags, &gen, &why)) {
        J->state = -1;
        J->log = why;
        return fail(PBN_EINVAL, "plan cannot be compiled: %s", why.c_str());
    }
    Nvrtc& N = nvrtc();
    if (!N.ok) {
        J->state = -1;
        J->log = N.err;
        return fail(PBN_ECUDA, "NVRTC unavailable: %s", N.err.c_str());
    }
    auto t0 = std::chrono::steady_clock::now();
    nvrtcProgram_t prog = nullptr;
    const char* hdrs[] = {kDeviceHeader};
    const char* hnames[] = {"pbn_device.cuh"};
    if (N.create(&prog, gen.src.c_str(), "pbn_plan_kernel.cu", 1, hdrs, hnames) != 0) {
        J->state = -1;
        J->log = "nvrtcCreateProgram failed";
        return fail(PBN_ECUDA, "nvrtcCreateProgram failed");
    }
    /* the warp-split form's long straight-line warp code: ptxas's default schedule
     * spends every register on overlap (and spills under a tight occupancy bound);
     * PBN_COMPILE_WS_O1 asks for -O1, which keeps fewer values live but overlaps less
     * (on the scale-free network the default schedule ran faster at every warp
     * count) */
    const char* opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", "-lineinfo", "--ptxas-options=-O1"};
    const bool o1 = (flags & PBN_COMPILE_WARP_SPLIT) && (flags & PBN_COMPILE_WS_O1);
    const int rc = N.compile(prog, o1 ? 4 : 3, opts);
    size_t ls = 0;
    N.log_size(prog, &ls);
    std::string log(ls, '\0');
    if (ls) N.log(prog, &log[0]);
    if (rc != 0) {
        N.destroy(&prog);
        J->state = -1;
        J->log = log;
        return fail(PBN_ECUDA, "NVRTC compilation failed: %.400s", log.c_str());
    }
    size_t cs = 0;
    N.cubin_size(prog, &cs);
    std::vector<char> cubin(cs);
    N.cubin(prog, cubin.data());
    N.destroy(&prog);
    cudaError_t e = cudaLibraryLoadData(&J->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&J->kern, J->lib, "pbn_plan_kernel");
    if (e != cudaSuccess) {
        J->state = -1;
        J->log = cudaGetErrorString(e);
        return fail(PBN_ECUDA, "loading the compiled plan failed: %s", cudaGetErrorString(e));
    }
    J->tab_bytes = gen.tab_bytes;
    J->warps = gen.warps;
    J->dyn_smem = gen.dyn_smem;
    J->static_smem = gen.static_smem;
    J->src = std::move(gen.src);
    J->compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    J->state = 1;
    return PBN_OK;
}

uint32_t jit_current_flags(const pbn_plan* plan) {
    pbn_jit_state* J = jit_state(plan);
    std::lock_guard<std::mutex> g(J->mu);
    return J->state == 1 ? J->flags : 0u;
}

bool jit_ready(const pbn_plan* plan) {
    pbn_jit_state* J = jit_state(plan);
    std::lock_guard<std::mutex> g(J->mu);
    return J->state == 1;
}

int jit_launch(const pbn_plan* plan, pbn_jit_params* P, uint32_t n_traj, int sms, cudaStream_t st) {
    pbn_jit_state* J = jit_state(plan);
    if (!jit_ready(plan)) return fail(PBN_EINVAL, "plan is not compiled");
    P->tab_bytes = J->tab_bytes;
    uint64_t tpb, grid;
    if (J->warps) {
        /* warp split: 32 trajectories per CTA of `warps` warps */
        tpb = 32ull * J->warps;
        grid = (n_traj + 31) / 32;
    } else {
        uint64_t per_sm = (n_traj + (uint64_t)sms - 1) / (uint64_t)sms;
        tpb = ((per_sm + 31) / 32) * 32;
        if (tpb > 512) tpb = 512;
        if (tpb < 64) tpb = 64;
        grid = (n_traj + tpb - 1) / tpb;
    }
    void* args[] = {P};
    const size_t dyn = J->dyn_smem ? J->dyn_smem : J->tab_bytes;
    const int se = ensure_dyn_smem(reinterpret_cast<const void*>(J->kern), dyn, J->static_smem);
    if (se != 0) return fail(PBN_ECUDA, "compiled plan launch: %s", cudaGetErrorString(static_cast<cudaError_t>(se)));
    cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(J->kern), dim3((unsigned)grid), dim3((unsigned)tpb), args,
                                     dyn, st);
    if (e != cudaSuccess) return fail(PBN_ECUDA, "compiled plan launch: %s", cudaGetErrorString(e));
    return PBN_OK;
}

}  // namespace pbn

extern "C" int pbn_plan_compile(const pbn_plan* plan, uint32_t flags, double* compile_ms) {
    if (!plan) return pbn::fail(PBN_EINVAL, "pbn_plan_compile: NULL plan");
    if (flags & ~(PBN_COMPILE_PERT_UNROLLED | PBN_COMPILE_INTERLEAVED | PBN_COMPILE_PIPELINED | PBN_COMPILE_MAGIC_GATHER |
                  PBN_COMPILE_WIDE | PBN_COMPILE_WARP_SPLIT | PBN_COMPILE_WARPS(31) | PBN_COMPILE_MINCTAS(7) |
                  PBN_COMPILE_WS_BATCH(3) | PBN_COMPILE_WS_O1 | PBN_COMPILE_WS_SELSMEM))
        return pbn::fail(PBN_EINVAL, "pbn_plan_compile: unknown flags");
    if ((flags & (PBN_COMPILE_WARPS(31) | PBN_COMPILE_MINCTAS(7) | PBN_COMPILE_WS_BATCH(3) | PBN_COMPILE_WS_O1 |
                  PBN_COMPILE_WS_SELSMEM)) &&
        !(flags & PBN_COMPILE_WARP_SPLIT))
        return pbn::fail(PBN_EINVAL, "pbn_plan_compile: warp counts and CTAs per SM need PBN_COMPILE_WARP_SPLIT");
    const int rc = pbn::jit_compile(plan, flags);
    if (rc == PBN_OK && compile_ms) *compile_ms = pbn::jit_state(plan)->compile_ms;
    return rc;
}

extern "C" int pbn_plan_compiled_attrs(const pbn_plan* plan, uint32_t* regs, uint32_t* local_bytes, uint32_t* flags) {
    if (!plan) return pbn::fail(PBN_EINVAL, "pbn_plan_compiled_attrs: NULL plan");
    pbn_jit_state* J = pbn::jit_state(plan);
    std::lock_guard<std::mutex> g(J->mu);
    if (J->state != 1) return pbn::fail(PBN_EINVAL, "pbn_plan_compiled_attrs: the plan is not compiled");
    cudaFuncAttributes fa;
    const cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(J->kern));
    if (e != cudaSuccess) return pbn::fail(PBN_ECUDA, "cudaFuncGetAttributes: %s", cudaGetErrorString(e));
    if (regs) *regs = (uint32_t)fa.numRegs;
    if (local_bytes) *local_bytes = (uint32_t)fa.localSizeBytes;
    if (flags) *flags = J->flags;
    return PBN_OK;
}

extern "C" int pbn_plan_source(const pbn_plan* plan, uint32_t flags, char* dst, size_t cap, size_t* len) {
    if (!plan) return pbn::fail(PBN_EINVAL, "pbn_plan_source: NULL plan");
    Generated gen;
    std::string why;
    if (!generate(*plan, flags, &gen, &why)) return pbn::fail(PBN_EINVAL, "plan cannot be compiled: %s", why.c_str());
    if (len) *len = gen.src.size();
    if (dst) {
        if (cap < gen.src.size() + 1) return pbn::fail(PBN_EINVAL, "pbn_plan_source: need %zu bytes", gen.src.size() + 1);
        memcpy(dst, gen.src.c_str(), gen.src.size() + 1);
    }
    return PBN_OK;
}
