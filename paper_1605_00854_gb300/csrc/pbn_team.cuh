/*
 * pbn_team.cuh -- the team interpreter: Algorithm 5 (ParallelSimulation) with the
 * step semantics of Eq. 1 for wide states, shared by the single-network team kernel
 * (pbn_sim.cu) and the batched form.
 *
 * A team of K warps simulates 32 x TPL trajectories: lane l of every warp on
 * trajectories l, l + 32, ... (TPL per lane).  Its shared memory holds two state
 * buffers as [row][TPL][lane] (row W32 of each stays zero: padded input records
 * read it), the choice bytes of the SEL slots as [slot][TPL][lane] and a
 * perturbation flag per trajectory.  Every warp of a team walks the same plan
 * records in step, so the records are broadcast loads decoded once for the lane's
 * TPL trajectories, and a lane's state reads hit its own bank.  Per step:
 *   A. warp w draws the perturbation words w, w + K, ... of its trajectories
 *      (Sec. 3.2, Step 2), XORs the flips of retained nodes into the current state
 *      and sets the trajectory's flag; it draws the SEL blocks w, w + K, ... and
 *      stores their choices (integer thresholds); it clears its rows of the next
 *      state;
 *   B. for its unperturbed trajectories a lane evaluates groups w, w + K, ... of the
 *      evaluation order (Sec. 3.3, Step 3: combined choice, input pattern,
 *      merged-table entry) and ORs their bits into the next state; a perturbed
 *      trajectory's rows are copied (Eq. 1: no function is applied);
 *   C. warp 0 takes the meta-state indicator of the new state and updates the
 *      counts V, n01, n10, n11 (Sec. 4.2); the warps write trace snapshots.
 * A CTA barrier ends each phase.  Node-wise semantics are not run here.
 */
#ifndef PBN_TEAM_CUH
#define PBN_TEAM_CUH

#include "pbn_device.cuh"
#include "pbn_image.h"

/* Shared-memory bytes of one team of 32 x tpl trajectories: two state buffers of
 * W32 + 1 rows, the choice bytes of the 4 n_sel SEL slots and the perturbation
 * flags. */
__host__ __device__ inline uint32_t pbn_team_smem_bytes(uint32_t W32, uint32_t n_sel, uint32_t tpl) {
    return 128u * tpl * (2u * (W32 + 1u) + n_sel + 1u);
}

/* One team member: warp wt (0 <= wt < K) of a team whose shared memory starts at
 * `team`; `spec` is the staged plan image (the records, and the tables when
 * TAB_SMEM).  The lane's trajectories are lt0 + 32 j (j < TPL), those with bit j of
 * `act` set are real (the others compute on dummy columns and write nothing).
 * Every thread of the CTA calls this with the same P.n_steps (the CTA's barriers
 * are taken inside).  Returns the counts V, n01, n10, n11 of trajectory j in
 * out[4 j ...] for lanes of warp 0 (zero elsewhere). */
template <int TPL, bool TRACE, bool TAB_SMEM, class VT>
__device__ __forceinline__ void pbn_team_run(const VT& P, const uint8_t* spec, uint8_t* team, uint32_t K,
                                             uint32_t wt, uint32_t lane, uint64_t lt0, uint32_t act,
                                             uint32_t out[4 * TPL]) {
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

    constexpr uint32_t RS = 32u * TPL;     /* words of one state row (all trajectories) */
    const uint32_t W32 = P.W32;
    const uint32_t RW = RS * (W32 + 1u);   /* words of one state buffer */
    uint32_t* const X = reinterpret_cast<uint32_t*>(team);
    uint8_t* const CH = reinterpret_cast<uint8_t*>(X + 2u * RW) + lane; /* [4 n_sel][TPL][32] choice bytes */
    uint32_t* const PF = X + 2u * RW + RS * P.n_sel;                   /* [TPL][32] perturbation flags */
    const uint32_t npairs = (W32 + 1u) / 2u;
    auto traj = [&](int j) -> uint64_t { return P.traj_begin + lt0 + 32u * (uint32_t)j; };
    auto real = [&](int j) -> bool { return (act >> j) & 1u; };

    uint32_t cV[TPL], c01[TPL], c10[TPL], c11[TPL], zp[TPL];
#pragma unroll
    for (int j = 0; j < TPL; ++j) cV[j] = c01[j] = c10[j] = c11[j] = zp[j] = 0u;

    /* ---- initial state: both buffers (with their zero rows) cleared, then keyed
     *      INIT draws ORed in, or the stored state loaded ---- */
    for (uint32_t i = wt * 32u + lane; i < 2u * RW; i += 32u * K) X[i] = 0u;
    if (wt == 0) {
#pragma unroll
        for (int j = 0; j < TPL; ++j) PF[32u * j + lane] = 0u;
    }
    __syncthreads();
    if (P.init == 0) {
#pragma unroll
        for (int j = 0; j < TPL; ++j) {
            const pbn_philox_step ps = pbn_philox_begin(P, traj(j), 0);
            for (uint32_t w = wt; w < P.W; w += K) {
                const uint4 x = pbn_philox_draw(P, ps, (PBN_DOM_INIT << 28) | (w >> 1));
                uint64_t word = (w & 1u) ? (((uint64_t)x.w << 32) | x.z) : (((uint64_t)x.y << 32) | x.x);
                word &= RET[w];
                while (word) {
                    const uint32_t b = __ffsll((long long)word) - 1;
                    word &= word - 1;
                    const uint32_t p = POS[64 * w + b];
                    atomicOr(&X[(p >> 5) * RS + 32u * j + lane], 1u << (p & 31));
                }
            }
        }
    } else {
        for (uint32_t pr = wt; pr < npairs; pr += K) {
#pragma unroll
            for (int j = 0; j < TPL; ++j) {
                if (!real(j)) continue;
                const uint64_t v = P.state[(uint64_t)pr * P.n_traj + lt0 + 32u * j];
                X[(2u * pr) * RS + 32u * j + lane] = (uint32_t)v;
                if (2u * pr + 1u < W32) X[(2u * pr + 1u) * RS + 32u * j + lane] = (uint32_t)(v >> 32);
            }
        }
    }
    __syncthreads();

    /* meta-state indicator of trajectory j in a state buffer (warp 0) */
    auto meta_z = [&](const uint32_t* B, int j) -> uint32_t {
        uint32_t ok = 1u;
        for (uint32_t m = 0; m < P.n_meta_rows; ++m)
            ok &= ((B[P.meta_row[m] * RS + 32u * j + lane] & P.meta_mask[m]) == P.meta_val[m]) ? 1u : 0u;
        return ok;
    };
    if (wt == 0) {
#pragma unroll
        for (int j = 0; j < TPL; ++j) {
            zp[j] = meta_z(X, j);
            if (P.count_first) cV[j] += zp[j];
        }
    }

    const uint32_t nl = P.n & 63u;
    const uint64_t last_lanes = nl ? ((1ull << nl) - 1ull) : ~0ull;
    uint32_t cur = 0;

    for (uint32_t k = 0; k < P.n_steps; ++k) {
        const uint64_t t = P.step_begin + k;
        uint32_t* const Sc = X + cur * RW;
        uint32_t* const Sn = X + (cur ^ 1u) * RW;

        /* ---- A. perturbation and SEL draws, split over the warps ---- */
        for (uint32_t r = wt; r < W32; r += K) {
#pragma unroll
            for (int j = 0; j < TPL; ++j) Sn[r * RS + 32u * j + lane] = 0u;
        }
#pragma unroll
        for (int j = 0; j < TPL; ++j) {
            const pbn_philox_step ps = pbn_philox_begin(P, traj(j), t);
            auto flip = [&](uint32_t p) { atomicXor(&Sc[(p >> 5) * RS + 32u * j + lane], 1u << (p & 31)); };
            uint32_t any = 0;
            if (P.sampler != 0u) {
                /* geometric sampler: per word the first perturbed lane among the
                 * remaining ones, one 64-bit uniform per decision; word pairs split
                 * over the warps */
                const uint64_t* GEO = reinterpret_cast<const uint64_t*>(P.image + P.off_geo);
                for (uint32_t wp = wt; 2 * wp < P.W; wp += K) {
                    const uint4 x0 = pbn_philox_draw(P, ps, (PBN_DOM_GEO << 28) | (wp << 8));
                    for (uint32_t h2 = 0; h2 < 2 && 2 * wp + h2 < P.W; ++h2) {
                        const uint32_t w = 2 * wp + h2;
                        const bool last = w == P.W - 1;
                        uint64_t U = h2 ? (((uint64_t)x0.w << 32) | x0.z) : (((uint64_t)x0.y << 32) | x0.x);
                        if (U >= (last ? P.geo_last : P.geo_full)) continue;
                        const uint32_t L = (last && nl) ? nl : 64u;
                        uint32_t pos = 0, jj = 0;
                        for (;;) {
                            if (U >= __ldg(GEO + (L - pos - 1))) break;
                            uint32_t q = 0;
                            while (U >= __ldg(GEO + q)) ++q;
                            any = 1u;
                            const uint32_t b = pos + q;
                            if ((RET[w] >> b) & 1ull) flip(POS[64 * w + b]);
                            pos = b + 1;
                            if (pos >= L) break;
                            ++jj;
                            const uint4 x = pbn_philox_draw(P, ps, (PBN_DOM_GEO << 28) | (wp << 8) | jj);
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
            if (any) PF[32u * j + lane] = 1u;
            /* SEL blocks: each slot's uniform becomes the node's 0-based choice */
            for (uint32_t i = wt; i < P.n_sel; i += K) {
                const uint4 x = pbn_philox_draw(P, ps, (PBN_DOM_SEL << 28) | SELBLK[i]);
                const uint32_t u[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int l = 0; l < 4; ++l) {
                    const uint4 S = SELSLOT[l * P.n_sel + i]; /* t1, t2, n_thr, first */
                    uint32_t c;
                    if (S.z <= 2u) {
                        c = ((S.z >= 1u) & (u[l] >= S.x)) + ((S.z >= 2u) & (u[l] >= S.y));
                    } else {
                        c = 0;
                        for (uint32_t q2 = 0; q2 < S.z; ++q2) c += (u[l] >= THR[S.w + q2]) ? 1u : 0u;
                    }
                    CH[((4u * i + l) * TPL + j) * 32u] = (uint8_t)c;
                }
            }
        }
        __syncthreads();
        /* ---- B. next state: groups split over the warps, bits ORed in ---- */
        uint32_t pm = 0; /* bit j: trajectory j was perturbed this step */
#pragma unroll
        for (int j = 0; j < TPL; ++j) pm |= (PF[32u * j + lane] != 0u ? 1u : 0u) << j;
        if (pm != (1u << TPL) - 1u) {
            const uint8_t* const ScB = reinterpret_cast<const uint8_t*>(Sc + lane);
            /* input patterns of q inputs from chunked records `stride` chunks apart, for
             * the trajectories in `which`; a record's bits above 5 give the row's byte
             * offset in a 32-bit-row state, so row * 128 TPL bytes here, and the
             * trajectory's word 128 j bytes further */
            auto gather = [&](const uint4* ch, uint32_t q, uint32_t stride, uint32_t x[TPL]) {
#pragma unroll
                for (int j = 0; j < TPL; ++j) x[j] = 0u;
                for (uint32_t b0 = 0; b0 < q; b0 += 4) {
                    const uint4 R = *ch;
                    ch += stride;
                    const uint8_t* const a0 = ScB + (R.x & ~31u) * TPL;
                    const uint8_t* const a1 = ScB + (R.y & ~31u) * TPL;
                    const uint8_t* const a2 = ScB + (R.z & ~31u) * TPL;
                    const uint8_t* const a3 = ScB + (R.w & ~31u) * TPL;
#pragma unroll
                    for (int j = 0; j < TPL; ++j) {
                        const uint32_t v0 = *reinterpret_cast<const uint32_t*>(a0 + 128u * j);
                        const uint32_t v1 = *reinterpret_cast<const uint32_t*>(a1 + 128u * j);
                        const uint32_t v2 = *reinterpret_cast<const uint32_t*>(a2 + 128u * j);
                        const uint32_t v3 = *reinterpret_cast<const uint32_t*>(a3 + 128u * j);
                        uint32_t x4 = __funnelshift_r(v0, v0, R.x) & 1u;
                        x4 |= __funnelshift_r(v1, v1, R.y) & 2u;
                        x4 |= __funnelshift_r(v2, v2, R.z) & 4u;
                        x4 |= __funnelshift_r(v3, v3, R.w) & 8u;
                        x[j] |= x4 << b0;
                    }
                }
            };
            auto choice = [&](uint32_t s, int j) -> uint32_t { return CH[(s * TPL + j) * 32u]; };
            /* group gi: per trajectory the table word and bit offset of its entry; the
             * entry mask and the group's shift in its output word */
            auto lookup = [&](uint32_t gi, uint32_t tw[TPL], uint32_t tb[TPL], uint32_t& msk, uint32_t& sh) {
                const uint4 G = GROUPS[gi]; /* tab_off, in_chunk, mul_first, q|l2w|n_mul|shift */
                const uint32_t q = G.w & 0xFFu;
                const uint32_t l2w = (G.w >> 8) & 0xFFu;
                const uint32_t n_mul = (G.w >> 16) & 0xFFu;
                sh = G.w >> 24;
                if (l2w == PBN_IMG_SPLIT) {
                    /* split node: only the selected function's table (per trajectory) */
                    msk = 1u;
                    const uint32_t slot = MULTI[G.z].x;
#pragma unroll
                    for (int j = 0; j < TPL; ++j) {
                        const uint2 F = SUBS[G.x + 32u * choice(slot, j)];
                        const uint4* ch = INPUTS + (F.x & 0x7FFFFFFu);
                        const uint32_t qf = F.x >> 27;
                        const uint8_t* const bj = ScB + 128u * j;
                        uint32_t x = 0;
                        for (uint32_t b0 = 0; b0 < qf; b0 += 4) {
                            const uint4 R = *ch++;
                            const uint32_t v0 = *reinterpret_cast<const uint32_t*>(bj + (R.x & ~31u) * TPL);
                            const uint32_t v1 = *reinterpret_cast<const uint32_t*>(bj + (R.y & ~31u) * TPL);
                            const uint32_t v2 = *reinterpret_cast<const uint32_t*>(bj + (R.z & ~31u) * TPL);
                            const uint32_t v3 = *reinterpret_cast<const uint32_t*>(bj + (R.w & ~31u) * TPL);
                            uint32_t x4 = __funnelshift_r(v0, v0, R.x) & 1u;
                            x4 |= __funnelshift_r(v1, v1, R.y) & 2u;
                            x4 |= __funnelshift_r(v2, v2, R.z) & 4u;
                            x4 |= __funnelshift_r(v3, v3, R.w) & 8u;
                            x |= x4 << b0;
                        }
                        tw[j] = F.y + (x >> 5);
                        tb[j] = x & 31u;
                    }
                    return;
                }
                uint32_t c[TPL];
#pragma unroll
                for (int j = 0; j < TPL; ++j) c[j] = 0u;
                for (uint32_t m = 0; m < n_mul; ++m) {
                    const uint2 M = MULTI[G.z + 32u * m]; /* choice slot, radix */
#pragma unroll
                    for (int j = 0; j < TPL; ++j) c[j] += choice(M.x, j) * M.y;
                }
                uint32_t x[TPL];
                gather(INPUTS + G.y, q, 32u, x);
                msk = (2u << ((1u << l2w) - 1u)) - 1u;
#pragma unroll
                for (int j = 0; j < TPL; ++j) {
                    const uint32_t bo = ((c[j] << q) | x[j]) << l2w;
                    tw[j] = G.x + (bo >> 5);
                    tb[j] = bo & 31u;
                }
            };
            auto tab_word = [&](uint32_t i) -> uint32_t { return TAB_SMEM ? TAB[i] : __ldg(TAB + i); };
            /* NG groups at a time: their table loads are in flight together */
            constexpr int NG = TPL == 1 ? 4 : 2;
            uint32_t g = wt;
            for (; g + (NG - 1) * K < P.n_groups; g += NG * K) {
                uint32_t go[NG], tw[NG][TPL], tb[NG][TPL], msk[NG], sh[NG], v[NG][TPL];
#pragma unroll
                for (int i = 0; i < NG; ++i) {
                    go[i] = GORDER[g + i * K];
                    lookup(go[i] & 0xFFFFFu, tw[i], tb[i], msk[i], sh[i]);
                }
#pragma unroll
                for (int i = 0; i < NG; ++i) {
#pragma unroll
                    for (int j = 0; j < TPL; ++j) v[i][j] = tab_word(tw[i][j]);
                }
#pragma unroll
                for (int i = 0; i < NG; ++i) {
#pragma unroll
                    for (int j = 0; j < TPL; ++j)
                        if (!((pm >> j) & 1u))
                            atomicOr(&Sn[(go[i] >> 20) * RS + 32u * j + lane], ((v[i][j] >> tb[i][j]) & msk[i]) << sh[i]);
                }
            }
            for (; g < P.n_groups; g += K) {
                const uint32_t go = GORDER[g];
                uint32_t tw[TPL], tb[TPL], msk, sh;
                lookup(go & 0xFFFFFu, tw, tb, msk, sh);
#pragma unroll
                for (int j = 0; j < TPL; ++j)
                    if (!((pm >> j) & 1u))
                        atomicOr(&Sn[(go >> 20) * RS + 32u * j + lane], ((tab_word(tw[j]) >> tb[j]) & msk) << sh);
            }
        }
        if (pm) {
            for (uint32_t r = wt; r < W32; r += K) {
#pragma unroll
                for (int j = 0; j < TPL; ++j)
                    if ((pm >> j) & 1u) Sn[r * RS + 32u * j + lane] = Sc[r * RS + 32u * j + lane];
            }
        }
        __syncthreads();

        /* ---- C. counts and trace of the new state ---- */
        if (wt == 0) {
            const uint32_t cv = k >= P.kv0 ? 1u : 0u;
            const uint32_t cp = k >= P.kp0 ? 1u : 0u;
#pragma unroll
            for (int j = 0; j < TPL; ++j) {
                PF[32u * j + lane] = 0u;
                const uint32_t z = meta_z(Sn, j);
                cV[j] += cv & z;
                c11[j] += cp & zp[j] & z;
                c01[j] += cp & (zp[j] ^ 1u) & z;
                c10[j] += cp & zp[j] & (z ^ 1u);
                zp[j] = z;
            }
        }
        if (TRACE && (k + 1) % P.trace_stride == 0) {
            const uint64_t snap = (k + 1) / P.trace_stride - 1;
            for (uint32_t pr = wt; pr < npairs; pr += K) {
#pragma unroll
                for (int j = 0; j < TPL; ++j) {
                    if (!real(j)) continue;
                    const uint32_t lo = Sn[(2u * pr) * RS + 32u * j + lane];
                    const uint32_t hi = 2u * pr + 1u < W32 ? Sn[(2u * pr + 1u) * RS + 32u * j + lane] : 0u;
                    P.trace[(snap * npairs + pr) * P.n_traj + lt0 + 32u * j] = ((uint64_t)hi << 32) | lo;
                }
            }
        }
        __syncthreads();
        cur ^= 1u;
    }

    /* ---- epilogue: final state, per-trajectory counts ---- */
    const uint32_t* Sb = X + cur * RW;
    for (uint32_t pr = wt; pr < npairs; pr += K) {
#pragma unroll
        for (int j = 0; j < TPL; ++j) {
            if (!real(j)) continue;
            const uint32_t lo = Sb[(2u * pr) * RS + 32u * j + lane];
            const uint32_t hi = 2u * pr + 1u < W32 ? Sb[(2u * pr + 1u) * RS + 32u * j + lane] : 0u;
            P.state[(uint64_t)pr * P.n_traj + lt0 + 32u * j] = ((uint64_t)hi << 32) | lo;
        }
    }
#pragma unroll
    for (int j = 0; j < TPL; ++j) {
        if (wt == 0 && real(j) && P.counts) {
            const uint64_t nt = P.n_traj, ltj = lt0 + 32u * j;
            P.counts[0 * nt + ltj] += cV[j];
            P.counts[1 * nt + ltj] += P.pairs - c01[j] - c10[j] - c11[j];
            P.counts[2 * nt + ltj] += c01[j];
            P.counts[3 * nt + ltj] += c10[j];
            P.counts[4 * nt + ltj] += c11[j];
        }
        out[4 * j + 0] = cV[j];
        out[4 * j + 1] = c01[j];
        out[4 * j + 2] = c10[j];
        out[4 * j + 3] = c11[j];
    }
}

#endif
