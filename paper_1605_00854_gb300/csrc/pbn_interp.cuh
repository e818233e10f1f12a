/*
 * pbn_interp.cuh -- the interpreter's per-trajectory simulation loop (Algorithm 5,
 * ParallelSimulation, with the step semantics of Eq. 1), shared by the
 * single-network kernel (pbn_sim.cu) and the batched work-queue kernel
 * (pbn_batch.cu).
 *
 * Per CTA the staged plan image sits at the start of shared memory; each
 * trajectory slot owns two state buffers of W32 + 1 32-bit words (the last one
 * always zero; odd stride, so a warp reading one row of 32 slots hits 32 banks)
 * and a choice row of n_sel | 1 words (one choice byte per SEL slot, four per SEL
 * block).  With LG > 1 lanes per trajectory the lanes split the perturbation words
 * and SEL blocks and take the groups in the image's evaluation order (shape classes,
 * output words alternating within a class), ORing into the shared next-state words.
 * Per step:
 *   1. perturbation (Sec. 3.2, Step 2): every original 64-node word draws its
 *      Bernoulli(P / 2^32) lanes bit-sliced, most significant level first, and
 *      stops once every lane is decided or no later level can change the outcome.
 *      Any set lane means a perturbed step (leaves included, which replaces
 *      Algorithm 1's single draw); the set lanes of retained nodes are flipped.
 *   2. otherwise (Sec. 3.3, Step 3): the SEL blocks of the retained multi-function
 *      nodes are drawn; for every group the combined choice c (mixed radix), the
 *      input pattern x (4-input chunks) and the table entry T[c][x] give the
 *      group's new bits, ORed into the next state at the group's offset (cum).
 *      A split node evaluates only its selected function's own table.
 *   3. the meta-state indicator z of the new state updates V, n01, n10, n11.
 * With node-wise semantics (P.per_node) every step runs 2 and then 1, and a
 * perturbed retained node takes the negation of its old value instead of its
 * function's output.
 */
#ifndef PBN_INTERP_CUH
#define PBN_INTERP_CUH

#include "pbn_device.cuh"
#include "pbn_image.h"

template <int LG>
__device__ __forceinline__ uint32_t group_mask() {
    if (LG == 32) return 0xFFFFFFFFu;
    const uint32_t lane = threadIdx.x & 31u;
    return ((1u << LG) - 1u) << (lane & ~(uint32_t)(LG - 1));
}

template <int LG>
__device__ __forceinline__ void group_sync() {
    if (LG > 1) __syncwarp(group_mask<LG>());
}

template <int LG>
__device__ __forceinline__ void xor_bit(uint32_t* w, uint32_t bit) {
    if (LG == 1) *w ^= bit;
    else atomicXor(w, bit);
}

template <int LG>
__device__ __forceinline__ void or_bit(uint32_t* w, uint32_t bit) {
    if (LG == 1) *w |= bit;
    else atomicOr(w, bit);
}

/* Simulate one trajectory slot of a CTA for P.n_steps steps (Algorithm 5 with
 * Eq. 1 semantics): initial or loaded state, per-step perturbation, selection and
 * merged-table evaluation, meta-state counts; writes the final state and the
 * per-trajectory counts and returns the four counters (V, n01, n10, n11) in out[]
 * for the caller's pooled reduction.  `smem` holds the staged plan image; the
 * trajectory rows start at smem_state_off.  VT is any type with the fields of
 * the launch parameters (kernel parameters or a per-network descriptor). */
template <int LG, bool TRACE, bool TAB_SMEM, bool SPEC_SMEM, class VT>
__device__ __forceinline__ void pbn_interp_run(const VT& P, uint8_t* smem, uint32_t smem_state_off, uint32_t NT,
                                               uint32_t slot, uint32_t lane, uint64_t lt, bool active,
                                               uint32_t out[4]) {
    const uint8_t* SP = SPEC_SMEM ? smem : P.image; /* specs: staged copy or the global image */
    const uint2* WORDS = reinterpret_cast<const uint2*>(SP + P.off_words);
    const uint4* GROUPS = reinterpret_cast<const uint4*>(SP + P.off_groups);
    const uint2* MULTI = reinterpret_cast<const uint2*>(SP + P.off_multi);
    const uint4* SELSLOT = reinterpret_cast<const uint4*>(SP + P.off_selslot);
    const uint32_t* THR = reinterpret_cast<const uint32_t*>(SP + P.off_thr);
    const uint4* INPUTS = reinterpret_cast<const uint4*>(SP + P.off_inputs);
    const uint32_t* SELBLK = reinterpret_cast<const uint32_t*>(SP + P.off_selblk);
    const uint32_t* GORDER = reinterpret_cast<const uint32_t*>(SP + P.off_gorder);
    const uint32_t* WGROUPS = reinterpret_cast<const uint32_t*>(SP + P.off_wgroups);
    const uint2* SUBS = reinterpret_cast<const uint2*>(SP + P.off_subs);
    const uint64_t* RET = reinterpret_cast<const uint64_t*>(P.image + P.off_ret);
    const uint32_t* POS = reinterpret_cast<const uint32_t*>(P.image + P.off_pos);
    const uint32_t* TAB = TAB_SMEM ? reinterpret_cast<const uint32_t*>(smem + P.off_tables)
                                   : reinterpret_cast<const uint32_t*>(P.image + P.off_tables);

    const uint32_t W32 = P.W32;
    const uint32_t W32P = W32 + 1;            /* odd stride: row r of every slot in its own bank */
    const uint32_t CHP = P.n_sel | 1u;        /* odd stride of the choice rows (one word per SEL block) */
    uint32_t* SBASE = reinterpret_cast<uint32_t*>(smem + smem_state_off); /* [2][NT][W32P] */
    uint32_t* CBASE = SBASE + 2 * NT * W32P;                                 /* [NT][CHP] */

    const uint64_t traj = P.traj_begin + lt;

    uint32_t* const S0 = SBASE + slot * W32P;  /* buffer b at S0 + b * bufstride; row W32 stays 0 */
    const uint32_t bufstride = NT * W32P;
    uint32_t* const Ct = CBASE + slot * CHP;  /* byte 4 i + l: choice of SEL slot 4 i + l */
    const uint8_t* const Cb = reinterpret_cast<const uint8_t*>(Ct);
    uint32_t cur = 0;

    uint32_t cV = 0, c01 = 0, c10 = 0, c11 = 0;

    if (active) {
        /* ---- initial state (both buffers' zero rows cleared) ---- */
        for (uint32_t r = lane; r <= W32; r += LG) {
            S0[bufstride + r] = 0u;
            if (P.init == 0 || r == W32) S0[r] = 0u;
        }
        group_sync<LG>();
        if (P.init == 0) {
            const pbn_philox_step ps = pbn_philox_begin(P, traj, 0);
            for (uint32_t w = lane; w < P.W; w += LG) {
                const uint4 x = pbn_philox_draw(P, ps, (PBN_DOM_INIT << 28) | (w >> 1));
                uint64_t word = (w & 1u) ? (((uint64_t)x.w << 32) | x.z) : (((uint64_t)x.y << 32) | x.x);
                word &= RET[w];
                while (word) {
                    const uint32_t b = __ffsll((long long)word) - 1;
                    word &= word - 1;
                    const uint32_t ps_ = POS[64 * w + b];
                    or_bit<LG>(&S0[ps_ >> 5], 1u << (ps_ & 31));
                }
            }
        } else {
            for (uint32_t r = lane; r < W32; r += LG) {
                const uint64_t v = P.state[(uint64_t)(r >> 1) * P.n_traj + lt];
                S0[r] = (r & 1u) ? (uint32_t)(v >> 32) : (uint32_t)v;
            }
        }
        group_sync<LG>();

        /* meta-state indicator of a state buffer (read by lane 0 of the group) */
        auto meta_z = [&](const uint32_t* Sb) -> uint32_t {
            uint32_t ok = 1u;
            for (uint32_t m = 0; m < P.n_meta_rows; ++m)
                ok &= ((Sb[P.meta_row[m]] & P.meta_mask[m]) == P.meta_val[m]) ? 1u : 0u;
            return ok;
        };
        uint32_t zp = meta_z(S0);
        if (P.count_first) cV += zp;

        const uint32_t nl = P.n & 63u;
        const uint64_t last_lanes = nl ? ((1ull << nl) - 1ull) : ~0ull;

        for (uint32_t k = 0; k < P.n_steps; ++k) {
            const uint64_t t = P.step_begin + k;
            const pbn_philox_step ps = pbn_philox_begin(P, traj, t);
            uint32_t* Sc = S0 + cur * bufstride;
            uint32_t* Sn = S0 + (cur ^ 1u) * bufstride;

            /* ---- 1. perturbation: bit-sliced u < P, most significant level first,
             *         stopping once every lane of the word is decided; flip(pos) is
             *         called for every perturbed retained node ---- */
            auto perturb = [&](auto&& flip) -> uint32_t {
                uint32_t any_l = 0;
                if (P.sampler != 0u) {
                    /* geometric sampler: per word the first perturbed lane among the
                     * remaining ones, one 64-bit uniform per decision; one block
                     * decides a pair of words in the common (no perturbation) case */
                    const uint64_t* GEO = reinterpret_cast<const uint64_t*>(P.image + P.off_geo);
                    for (uint32_t wp = lane; 2 * wp < P.W; wp += LG) {
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
                                uint32_t k = 0;
                                while (U >= __ldg(GEO + k)) ++k;
                                any_l = 1u;
                                const uint32_t b = pos + k;
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
                    for (uint32_t w = lane; w < P.W; w += LG) {
                        const uint64_t valid = (w == P.W - 1) ? last_lanes : ~0ull;
                        uint32_t und_lo = (uint32_t)valid, und_hi = (uint32_t)(valid >> 32);
                        uint32_t pert_lo = 0, pert_hi = 0;
                        uint32_t pp = P.P; /* level 2h uses bit 31 of pp, level 2h+1 bit 30 */
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
                            any_l = 1u;
                            uint64_t f = ((((uint64_t)pert_hi) << 32) | pert_lo) & RET[w];
                            while (f) {
                                const uint32_t b = __ffsll((long long)f) - 1;
                                f &= f - 1;
                                flip(POS[64 * w + b]);
                            }
                        }
                    }
                }
                return any_l;
            };

            /* ---- 2. selection and merged-table evaluation: Sn from Sc ---- */
            auto select_eval = [&]() {
                /* ---- 2a. selection: draw the SEL blocks, turn each slot's uniform into
                 *          the node's 0-based choice (integer thresholds), one byte each ---- */
                auto choices = [&](const uint4 x, uint32_t i) -> uint32_t {
                    const uint32_t u[4] = {x.x, x.y, x.z, x.w};
                    uint32_t word = 0;
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
                        word |= j << (8 * l);
                    }
                    return word;
                };
                uint32_t i = lane;
                for (; i + LG < P.n_sel; i += 2 * LG) {
                    const uint4 x = pbn_philox_draw(P, ps, (PBN_DOM_SEL << 28) | SELBLK[i]);
                    const uint4 y = pbn_philox_draw(P, ps, (PBN_DOM_SEL << 28) | SELBLK[i + LG]);
                    Ct[i] = choices(x, i);
                    Ct[i + LG] = choices(y, i + LG);
                }
                if (i < P.n_sel) {
                    const uint4 x = pbn_philox_draw(P, ps, (PBN_DOM_SEL << 28) | SELBLK[i]);
                    Ct[i] = choices(x, i);
                }
                group_sync<LG>();
                /* ---- 2b. merged-table evaluation ---- */
                const uint8_t* Sc8 = reinterpret_cast<const uint8_t*>(Sc);
                /* input pattern of q inputs from their chunked records (chunks
                 * `stride` apart: 32 in the row-interleaved group layout, 1 for the
                 * functions of a split node) */
                auto gather = [&](const uint4* ch, uint32_t q, uint32_t stride) -> uint32_t {
                    uint32_t x = 0;
                    for (uint32_t b0 = 0; b0 < q; b0 += 4) {
                        const uint4 R = *ch;
                        ch += stride;
                        const uint32_t v0 = *reinterpret_cast<const uint32_t*>(Sc8 + (R.x >> 5));
                        const uint32_t v1 = *reinterpret_cast<const uint32_t*>(Sc8 + (R.y >> 5));
                        const uint32_t v2 = *reinterpret_cast<const uint32_t*>(Sc8 + (R.z >> 5));
                        const uint32_t v3 = *reinterpret_cast<const uint32_t*>(Sc8 + (R.w >> 5));
                        uint32_t x4 = __funnelshift_r(v0, v0, R.x) & 1u;
                        x4 |= __funnelshift_r(v1, v1, R.y) & 2u;
                        x4 |= __funnelshift_r(v2, v2, R.z) & 4u;
                        x4 |= __funnelshift_r(v3, v3, R.w) & 8u;
                        x |= x4 << b0;
                    }
                    return x;
                };
                /* where group gi's entry lies: table word, bit offset, entry mask and
                 * the group's shift in its output word */
                auto group_lookup = [&](uint32_t gi) -> uint4 {
                    const uint4 G = GROUPS[gi]; /* tab_off, in_chunk, mul_first, q|l2w|n_mul|shift */
                    const uint32_t q = G.w & 0xFFu;
                    const uint32_t l2w = (G.w >> 8) & 0xFFu;
                    const uint32_t n_mul = (G.w >> 16) & 0xFFu;
                    const uint32_t shift = G.w >> 24;
                    if (l2w == PBN_IMG_SPLIT) {
                        /* split node: only the selected function is evaluated */
                        const uint2 F = SUBS[G.x + 32u * Cb[MULTI[G.z].x]]; /* in_chunk | k << 27, tab_off */
                        const uint32_t x = gather(INPUTS + (F.x & 0x7FFFFFFu), F.x >> 27, 1u);
                        return make_uint4(F.y + (x >> 5), x & 31u, 1u, shift);
                    }
                    uint32_t c = 0;
                    for (uint32_t m = 0; m < n_mul; ++m) {
                        const uint2 M = MULTI[G.z + 32u * m]; /* choice byte, radix */
                        c += (uint32_t)Cb[M.x] * M.y;
                    }
                    const uint32_t x = gather(INPUTS + G.y, q, 32u);
                    const uint32_t bo = ((c << q) | x) << l2w;
                    return make_uint4(G.x + (bo >> 5), bo & 31u, (2u << ((1u << l2w) - 1u)) - 1u, shift);
                };
                auto tab_word = [&](uint32_t i) -> uint32_t { return TAB_SMEM ? TAB[i] : __ldg(TAB + i); };
                auto entry_bits = [&](const uint4 L, uint32_t tw) -> uint32_t { return ((tw >> L.y) & L.z) << L.w; };
                /* new bits of group gi, already at their place in the output word */
                auto group_bits = [&](uint32_t gi) -> uint32_t {
                    const uint4 L = group_lookup(gi);
                    return entry_bits(L, tab_word(L.x));
                };
                if (LG == 1) {
                    /* word by word, the word's groups ORed in a register */
                    for (uint32_t w = 0; w < W32; ++w) {
                        const uint2 wr = WORDS[w];
                        uint32_t acc = 0;
                        for (uint32_t i = wr.x; i < wr.x + wr.y; ++i) acc |= group_bits(WGROUPS[i]);
                        Sn[w] = acc;
                    }
                } else {
                    /* the lanes of a trajectory take the groups in shape order (so they
                     * run in step) and OR their bits into the shared next-state words */
                    for (uint32_t w = lane; w < W32; w += LG) Sn[w] = 0u;
                    group_sync<LG>();
                    /* four groups per lane at a time: their table loads are in flight
                     * together (they dominate when the tables are in L2) */
                    uint32_t k = lane;
                    for (; k + 3 * LG < P.n_groups; k += 4 * LG) {
                        uint32_t go[4], tw[4];
                        uint4 L[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            go[i] = GORDER[k + i * LG];
                            L[i] = group_lookup(go[i] & 0xFFFFFu);
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) tw[i] = tab_word(L[i].x);
#pragma unroll
                        for (int i = 0; i < 4; ++i) atomicOr(&Sn[go[i] >> 20], entry_bits(L[i], tw[i]));
                    }
                    for (; k < P.n_groups; k += LG) {
                        const uint32_t go = GORDER[k];
                        atomicOr(&Sn[go >> 20], group_bits(go & 0xFFFFFu));
                    }
                }
                group_sync<LG>();
            };

            if (!P.per_node) {
                /* Eq. 1: any perturbed node (leaves included) flips the perturbed
                 * retained nodes and no function is applied */
                const uint32_t any_l = perturb([&](uint32_t ps_) { xor_bit<LG>(&Sc[ps_ >> 5], 1u << (ps_ & 31)); });
                uint32_t any = any_l;
                if (LG > 1) {
                    group_sync<LG>();
                    any = (__ballot_sync(group_mask<LG>(), any_l) & group_mask<LG>()) ? 1u : 0u;
                }
                if (!any) {
                    select_eval();
                    cur ^= 1u;
                }
            } else {
                /* node-wise: every node applies its function, then each perturbed
                 * node takes the negation of its old value instead */
                select_eval();
                perturb([&](uint32_t ps_) {
                    uint32_t* wn = &Sn[ps_ >> 5];
                    const uint32_t m = ~(*wn ^ Sc[ps_ >> 5]) & (1u << (ps_ & 31));
                    if (m) xor_bit<LG>(wn, m);
                });
                group_sync<LG>();
                cur ^= 1u;
            }

            /* ---- 3. meta-state counts ---- */
            if (lane == 0) {
                const uint32_t* Sb = S0 + cur * bufstride;
                const uint32_t z = meta_z(Sb);
                const uint32_t cv = k >= P.kv0 ? 1u : 0u;
                const uint32_t cp = k >= P.kp0 ? 1u : 0u;
                cV += cv & z;
                c11 += cp & zp & z;
                c01 += cp & (zp ^ 1u) & z;
                c10 += cp & zp & (z ^ 1u);
                zp = z;
                if (TRACE && (k + 1) % P.trace_stride == 0) {
                    const uint64_t snap = (k + 1) / P.trace_stride - 1;
                    for (uint32_t r = 0; r < W32; r += 2) {
                        const uint64_t v = ((uint64_t)Sb[r + 1] << 32) | Sb[r];
                        P.trace[(snap * (W32 / 2) + r / 2) * P.n_traj + lt] = v;
                    }
                }
            }
            group_sync<LG>();
        }

        /* ---- epilogue: state and counts ---- */
        const uint32_t* Sb = S0 + cur * bufstride;
        for (uint32_t r = lane * 2; r < W32; r += 2 * LG) {
            const uint64_t v = ((uint64_t)Sb[r + 1] << 32) | Sb[r];
            P.state[(uint64_t)(r >> 1) * P.n_traj + lt] = v;
        }
        if (lane == 0 && P.counts) {
            const uint32_t c00 = P.pairs - c01 - c10 - c11;
            const uint64_t nt = P.n_traj;
            P.counts[0 * nt + lt] += cV;
            P.counts[1 * nt + lt] += c00;
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
