/*
 * pbn_team.cuh -- the team interpreter: Algorithm 5 (ParallelSimulation) with the
 * step semantics of Eq. 1 for wide states, shared by the single-network team kernel
 * (pbn_sim.cu) and the batched form.
 *
 * A team of K warps simulates 32 trajectories, lane l of every warp on trajectory
 * l.  Its shared memory holds two state buffers as [row][lane] (row W32 of each
 * stays zero: padded input records read it), the choice bytes of the SEL slots as
 * [slot][lane] and a perturbation flag per lane.  Every warp of a team walks the
 * same plan records in step, so the records are broadcast loads and a lane's state
 * reads hit its own bank.  Per step:
 *   A. warp w draws the perturbation words w, w + K, ... of its 32 trajectories
 *      (Sec. 3.2, Step 2), XORs the flips of retained nodes into the current state
 *      and sets the lane's flag; it draws the SEL blocks w, w + K, ... and stores
 *      their choices (integer thresholds); it clears its rows of the next state;
 *   B. an unperturbed lane evaluates groups w, w + K, ... of the evaluation order
 *      (Sec. 3.3, Step 3: combined choice, input pattern, merged-table entry) and
 *      ORs their bits into the next state; a perturbed lane copies its rows
 *      (Eq. 1: no function is applied);
 *   C. warp 0 takes the meta-state indicator of the new state and updates the
 *      counts V, n01, n10, n11 (Sec. 4.2); the warps write trace snapshots.
 * A CTA barrier ends each phase.  Node-wise semantics are not run here.
 */
#ifndef PBN_TEAM_CUH
#define PBN_TEAM_CUH

#include "pbn_device.cuh"
#include "pbn_image.h"

/* Shared-memory bytes of one team: two state buffers of W32 + 1 rows, the choice
 * bytes of the 4 n_sel SEL slots, 32 lanes each, and the perturbation flags. */
__host__ __device__ inline uint32_t pbn_team_smem_bytes(uint32_t W32, uint32_t n_sel) {
    return 128u * (2u * (W32 + 1u) + n_sel + 1u);
}

/* One team member: warp wt (0 <= wt < K) of a team whose shared memory starts at
 * `team`; `spec` is the staged plan image (the records, and the tables when
 * TAB_SMEM).  Every thread of the CTA calls this with the same P.n_steps (the CTA's
 * barriers are taken inside); lanes with `active` false compute on a dummy column
 * and write nothing.  Returns the counts V, n01, n10, n11 in out[] for lanes of
 * warp 0 (zero elsewhere). */
template <bool TRACE, bool TAB_SMEM, class VT>
__device__ __forceinline__ void pbn_team_run(const VT& P, const uint8_t* spec, uint8_t* team, uint32_t K,
                                             uint32_t wt, uint32_t lane, uint64_t lt, bool active, uint32_t out[4]) {
    const uint4* GROUPS = reinterpret_cast<const uint4*>(spec + P.off_groups);
    const uint2* MULTI = reinterpret_cast<const uint2*>(spec + P.off_multi);
    const uint4* SELSLOT = reinterpret_cast<const uint4*>(spec + P.off_selslot);
    const uint32_t* THR = reinterpret_cast<const uint32_t*>(spec + P.off_thr);
    const uint4* INPUTS = reinterpret_cast<const uint4*>(spec + P.off_inputs);
    const uint32_t* SELBLK = reinterpret_cast<const uint32_t*>(spec + P.off_selblk);
    const uint32_t* GORDER = reinterpret_cast<const uint32_t*>(spec + P.off_gorder);
    const uint2* SUBS = reinterpret_cast<const uint2*>(spec + P.off_subs);
    const uint64_t* RET = reinterpret_cast<const uint64_t*>(P.image + P.off_ret);
    const uint32_t* POS = reinterpret_cast<const uint32_t*>(P.image + P.off_pos);
    const uint32_t* TAB = TAB_SMEM ? reinterpret_cast<const uint32_t*>(spec + P.off_tables)
                                   : reinterpret_cast<const uint32_t*>(P.image + P.off_tables);

    const uint32_t W32 = P.W32;
    const uint32_t RW = 32u * (W32 + 1u); /* words of one state buffer */
    uint32_t* const X = reinterpret_cast<uint32_t*>(team);
    uint8_t* const CH = reinterpret_cast<uint8_t*>(X + 2u * RW) + lane; /* [4 n_sel][32] choice bytes */
    uint32_t* const PF = X + 2u * RW + 32u * P.n_sel;                  /* [32] perturbation flags */
    const uint64_t traj = P.traj_begin + lt;
    const uint32_t npairs = (W32 + 1u) / 2u;

    uint32_t cV = 0, c01 = 0, c10 = 0, c11 = 0;

    /* ---- initial state: both buffers (with their zero rows) cleared, then keyed
     *      INIT draws ORed in, or the stored state loaded ---- */
    for (uint32_t i = wt * 32u + lane; i < 2u * RW; i += 32u * K) X[i] = 0u;
    if (wt == 0) PF[lane] = 0u;
    __syncthreads();
    if (P.init == 0) {
        const pbn_philox_step ps = pbn_philox_begin(P, traj, 0);
        for (uint32_t w = wt; w < P.W; w += K) {
            const uint4 x = pbn_philox_draw(P, ps, (PBN_DOM_INIT << 28) | (w >> 1));
            uint64_t word = (w & 1u) ? (((uint64_t)x.w << 32) | x.z) : (((uint64_t)x.y << 32) | x.x);
            word &= RET[w];
            while (word) {
                const uint32_t b = __ffsll((long long)word) - 1;
                word &= word - 1;
                const uint32_t p = POS[64 * w + b];
                atomicOr(&X[(p >> 5) * 32u + lane], 1u << (p & 31));
            }
        }
    } else if (active) {
        for (uint32_t pr = wt; pr < npairs; pr += K) {
            const uint64_t v = P.state[(uint64_t)pr * P.n_traj + lt];
            X[(2u * pr) * 32u + lane] = (uint32_t)v;
            if (2u * pr + 1u < W32) X[(2u * pr + 1u) * 32u + lane] = (uint32_t)(v >> 32);
        }
    }
    __syncthreads();

    /* meta-state indicator of a state buffer for this lane's trajectory (warp 0) */
    auto meta_z = [&](const uint32_t* B) -> uint32_t {
        uint32_t ok = 1u;
        for (uint32_t m = 0; m < P.n_meta_rows; ++m)
            ok &= ((B[P.meta_row[m] * 32u + lane] & P.meta_mask[m]) == P.meta_val[m]) ? 1u : 0u;
        return ok;
    };
    uint32_t zp = 0;
    if (wt == 0) {
        zp = meta_z(X);
        if (P.count_first) cV += zp;
    }

    const uint32_t nl = P.n & 63u;
    const uint64_t last_lanes = nl ? ((1ull << nl) - 1ull) : ~0ull;
    uint32_t cur = 0;

    for (uint32_t k = 0; k < P.n_steps; ++k) {
        const uint64_t t = P.step_begin + k;
        const pbn_philox_step ps = pbn_philox_begin(P, traj, t);
        uint32_t* const Sc = X + cur * RW;
        uint32_t* const Sn = X + (cur ^ 1u) * RW;

        /* ---- A. perturbation and SEL draws, split over the warps ---- */
        for (uint32_t r = wt; r < W32; r += K) Sn[r * 32u + lane] = 0u;
        auto flip = [&](uint32_t p) { atomicXor(&Sc[(p >> 5) * 32u + lane], 1u << (p & 31)); };
        uint32_t any = 0;
        if (P.sampler != 0u) {
            /* geometric sampler: per word the first perturbed lane among the remaining
             * ones, one 64-bit uniform per decision; word pairs split over the warps */
            const uint64_t* GEO = reinterpret_cast<const uint64_t*>(P.image + P.off_geo);
            for (uint32_t wp = wt; 2 * wp < P.W; wp += K) {
                const uint4 x0 = pbn_philox_draw(P, ps, (PBN_DOM_GEO << 28) | (wp << 8));
                for (uint32_t h2 = 0; h2 < 2 && 2 * wp + h2 < P.W; ++h2) {
                    const uint32_t w = 2 * wp + h2;
                    const bool last = w == P.W - 1;
                    uint64_t U = h2 ? (((uint64_t)x0.w << 32) | x0.z) : (((uint64_t)x0.y << 32) | x0.x);
                    if (U >= (last ? P.geo_last : P.geo_full)) continue;
                    const uint32_t L = (last && nl) ? nl : 64u;
                    uint32_t pos = 0, j = 0;
                    for (;;) {
                        if (U >= __ldg(GEO + (L - pos - 1))) break;
                        uint32_t q = 0;
                        while (U >= __ldg(GEO + q)) ++q;
                        any = 1u;
                        const uint32_t b = pos + q;
                        if ((RET[w] >> b) & 1ull) flip(POS[64 * w + b]);
                        pos = b + 1;
                        if (pos >= L) break;
                        ++j;
                        const uint4 x = pbn_philox_draw(P, ps, (PBN_DOM_GEO << 28) | (wp << 8) | j);
                        U = h2 ? (((uint64_t)x.w << 32) | x.z) : (((uint64_t)x.y << 32) | x.x);
                    }
                }
            }
        } else if (P.P != 0u) {
            /* bit-sliced u < P per 64-node word, most significant level first */
            for (uint32_t w = wt; w < P.W; w += K) {
                const uint64_t valid = (w == P.W - 1) ? last_lanes : ~0ull;
                uint32_t und_lo = (uint32_t)valid, und_hi = (uint32_t)(valid >> 32);
                uint32_t pert_lo = 0, pert_hi = 0;
                uint32_t pp = P.P;
                for (uint32_t h = 0; h < P.hmax && (und_lo | und_hi); ++h) {
                    const uint4 x = pbn_philox_draw(P, ps, (PBN_DOM_PERT << 28) | (w << 4) | h);
                    const uint32_t m0 = (uint32_t)((int32_t)pp >> 31);
                    const uint32_t m1 = (uint32_t)((int32_t)(pp << 1) >> 31);
                    pp <<= 2;
                    pert_lo |= und_lo & ~x.x & m0;
                    pert_hi |= und_hi & ~x.y & m0;
                    und_lo &= ~(x.x ^ m0);
                    und_hi &= ~(x.y ^ m0);
                    pert_lo |= und_lo & ~x.z & m1;
                    pert_hi |= und_hi & ~x.w & m1;
                    und_lo &= ~(x.z ^ m1);
                    und_hi &= ~(x.w ^ m1);
                }
                if (pert_lo | pert_hi) {
                    any = 1u;
                    uint64_t f = ((((uint64_t)pert_hi) << 32) | pert_lo) & RET[w];
                    while (f) {
                        const uint32_t b = __ffsll((long long)f) - 1;
                        f &= f - 1;
                        flip(POS[64 * w + b]);
                    }
                }
            }
        }
        if (any) PF[lane] = 1u;
        /* SEL blocks: each slot's uniform becomes the node's 0-based choice */
        for (uint32_t i = wt; i < P.n_sel; i += K) {
            const uint4 x = pbn_philox_draw(P, ps, (PBN_DOM_SEL << 28) | SELBLK[i]);
            const uint32_t u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const uint4 S = SELSLOT[l * P.n_sel + i]; /* t1, t2, n_thr, first */
                uint32_t j;
                if (S.z <= 2u) {
                    j = ((S.z >= 1u) & (u[l] >= S.x)) + ((S.z >= 2u) & (u[l] >= S.y));
                } else {
                    j = 0;
                    for (uint32_t q2 = 0; q2 < S.z; ++q2) j += (u[l] >= THR[S.w + q2]) ? 1u : 0u;
                }
                CH[(4u * i + l) * 32u] = (uint8_t)j;
            }
        }
        __syncthreads();

        /* ---- B. next state: groups split over the warps, bits ORed in ---- */
        if (PF[lane] == 0u) {
            const uint8_t* const ScB = reinterpret_cast<const uint8_t*>(Sc + lane);
            /* input pattern of q inputs from chunked records `stride` chunks apart; a
             * record's bits above 5 give the row's byte offset in a 32-bit-row state,
             * so row * 128 bytes here */
            auto gather = [&](const uint4* ch, uint32_t q, uint32_t stride) -> uint32_t {
                uint32_t x = 0;
                for (uint32_t b0 = 0; b0 < q; b0 += 4) {
                    const uint4 R = *ch;
                    ch += stride;
                    const uint32_t v0 = *reinterpret_cast<const uint32_t*>(ScB + (R.x & ~31u));
                    const uint32_t v1 = *reinterpret_cast<const uint32_t*>(ScB + (R.y & ~31u));
                    const uint32_t v2 = *reinterpret_cast<const uint32_t*>(ScB + (R.z & ~31u));
                    const uint32_t v3 = *reinterpret_cast<const uint32_t*>(ScB + (R.w & ~31u));
                    uint32_t x4 = __funnelshift_r(v0, v0, R.x) & 1u;
                    x4 |= __funnelshift_r(v1, v1, R.y) & 2u;
                    x4 |= __funnelshift_r(v2, v2, R.z) & 4u;
                    x4 |= __funnelshift_r(v3, v3, R.w) & 8u;
                    x |= x4 << b0;
                }
                return x;
            };
            auto choice = [&](uint32_t s) -> uint32_t { return CH[s * 32u]; };
            /* table word, bit offset and entry mask of group gi, and its shift */
            auto lookup = [&](uint32_t gi) -> uint4 {
                const uint4 G = GROUPS[gi]; /* tab_off, in_chunk, mul_first, q|l2w|n_mul|shift */
                const uint32_t q = G.w & 0xFFu;
                const uint32_t l2w = (G.w >> 8) & 0xFFu;
                const uint32_t n_mul = (G.w >> 16) & 0xFFu;
                const uint32_t shift = G.w >> 24;
                if (l2w == PBN_IMG_SPLIT) {
                    /* split node: only the selected function's table */
                    const uint2 F = SUBS[G.x + 32u * choice(MULTI[G.z].x)];
                    const uint32_t x = gather(INPUTS + (F.x & 0x7FFFFFFu), F.x >> 27, 1u);
                    return make_uint4(F.y + (x >> 5), x & 31u, 1u, shift);
                }
                uint32_t c = 0;
                for (uint32_t m = 0; m < n_mul; ++m) {
                    const uint2 M = MULTI[G.z + 32u * m]; /* choice slot, radix */
                    c += choice(M.x) * M.y;
                }
                const uint32_t x = gather(INPUTS + G.y, q, 32u);
                const uint32_t bo = ((c << q) | x) << l2w;
                return make_uint4(G.x + (bo >> 5), bo & 31u, (2u << ((1u << l2w) - 1u)) - 1u, shift);
            };
            auto tab_word = [&](uint32_t i) -> uint32_t { return TAB_SMEM ? TAB[i] : __ldg(TAB + i); };
            uint32_t g = wt;
            /* four groups at a time: their table loads are in flight together */
            for (; g + 3u * K < P.n_groups; g += 4u * K) {
                uint32_t go[4], tw[4];
                uint4 L[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    go[i] = GORDER[g + i * K];
                    L[i] = lookup(go[i] & 0xFFFFFu);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) tw[i] = tab_word(L[i].x);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    atomicOr(&Sn[(go[i] >> 20) * 32u + lane], ((tw[i] >> L[i].y) & L[i].z) << L[i].w);
            }
            for (; g < P.n_groups; g += K) {
                const uint32_t go = GORDER[g];
                const uint4 L = lookup(go & 0xFFFFFu);
                atomicOr(&Sn[(go >> 20) * 32u + lane], ((tab_word(L.x) >> L.y) & L.z) << L.w);
            }
        } else {
            for (uint32_t r = wt; r < W32; r += K) Sn[r * 32u + lane] = Sc[r * 32u + lane];
        }
        __syncthreads();

        /* ---- C. counts and trace of the new state ---- */
        if (wt == 0) {
            PF[lane] = 0u;
            const uint32_t z = meta_z(Sn);
            const uint32_t cv = k >= P.kv0 ? 1u : 0u;
            const uint32_t cp = k >= P.kp0 ? 1u : 0u;
            cV += cv & z;
            c11 += cp & zp & z;
            c01 += cp & (zp ^ 1u) & z;
            c10 += cp & zp & (z ^ 1u);
            zp = z;
        }
        if (TRACE && active && (k + 1) % P.trace_stride == 0) {
            const uint64_t snap = (k + 1) / P.trace_stride - 1;
            for (uint32_t pr = wt; pr < npairs; pr += K) {
                const uint32_t lo = Sn[(2u * pr) * 32u + lane];
                const uint32_t hi = 2u * pr + 1u < W32 ? Sn[(2u * pr + 1u) * 32u + lane] : 0u;
                P.trace[(snap * npairs + pr) * P.n_traj + lt] = ((uint64_t)hi << 32) | lo;
            }
        }
        __syncthreads();
        cur ^= 1u;
    }

    /* ---- epilogue: final state, per-trajectory counts ---- */
    if (active) {
        const uint32_t* Sb = X + cur * RW;
        for (uint32_t pr = wt; pr < npairs; pr += K) {
            const uint32_t lo = Sb[(2u * pr) * 32u + lane];
            const uint32_t hi = 2u * pr + 1u < W32 ? Sb[(2u * pr + 1u) * 32u + lane] : 0u;
            P.state[(uint64_t)pr * P.n_traj + lt] = ((uint64_t)hi << 32) | lo;
        }
        if (wt == 0 && P.counts) {
            const uint64_t nt = P.n_traj;
            P.counts[0 * nt + lt] += cV;
            P.counts[1 * nt + lt] += P.pairs - c01 - c10 - c11;
            P.counts[2 * nt + lt] += c01;
            P.counts[3 * nt + lt] += c10;
            P.counts[4 * nt + lt] += c11;
        }
    }
    out[0] = cV;
    out[1] = c01;
    out[2] = c10;
    out[3] = c11;
}

#endif
