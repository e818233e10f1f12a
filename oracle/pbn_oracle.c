/*
 * pbn_oracle.c -- plain, slow, obviously-correct CPU oracle for PBN simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only tests/, __graft_entry__.smoke() and the CPU-baseline leg of
 * bench.py use it.  It shares no code, header, table or constant generator with
 * the CUDA/C++ library: it parses the network text itself, runs its own Philox,
 * computes its own thresholds, and simulates the UNREDUCED, UNGROUPED network.
 *
 * What it computes (paper section / equation in brackets):
 *   - the PBN model G(X,F) with selection probabilities C_i            [Sec. 2.1]
 *   - one step of the perturbed PBN, Eq. 1: draw gamma_i ~ Bernoulli(p)
 *     for every node; if gamma != 0 the next state is s XOR gamma, otherwise
 *     every node applies a predictor function chosen by C_i             [Eq. 1]
 *   - the node-wise variant (semantics 1): node i takes NOT s_i if gamma_i = 1
 *     and its selected predictor function's value otherwise, whatever the
 *     other nodes draw                                 [Sec. 2.1, node-wise reading]
 *   - the meta-state visit / transition counts of the two-state Markov
 *     chain estimator, taken over a counting window                     [Sec. 4.2]
 *   - the exact transition matrix of the ergodic DTMC for tiny n          [Sec. 2.1]
 *   - the leaf set of Definition 1                                        [Sec. 3.1, Def. 1]
 *
 * Random draws follow the keyed contract (the paper uses an unspecified rand()
 * and alias tables; the keyed contract is this project's reading):
 *   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = 64-bit seed
 *   (k0 = low half, k1 = high half), counter
 *     c0 = trajectory id bits 0..31, c1 = step bits 0..31,
 *     c2 = step bits 32..47 | trajectory id bits 32..47 << 16,
 *     c3 = domain << 28 | index.
 *   PERT (domain 1): node i = 64w + b.  Index w << 4 | h gives levels 2h
 *     (x1:x0) and 2h+1 (x3:x2).  u_i is the 32-bit number whose bit 31-l is
 *     bit b of level l.  gamma_i = [u_i < P], P = floor(p * 2^32).
 *   SEL (domain 2): nodes with >= 2 functions ranked by ascending id; rank r
 *     takes word x_{r mod 4} of index r / 4 as u.  Choice (0-based) is the
 *     number of j in 1..l-1 with u >= T_j, T_j = min(floor(C_j 2^32), 2^32),
 *     C_j = C_{j-1} + c_j summed left to right in fp64.
 *   INIT (domain 3, step 0): word w of s(0) is x1:x0 of index w/2 if w is
 *     even, x3:x2 otherwise; bit b is node 64w + b.
 *   GEO (domain 4, the second perturbation sampler): for 64-node word w with L
 *     valid lanes, decisions j = 0, 1, ... take the 64-bit U_j = x1:x0 (w even)
 *     or x3:x2 (w odd) of index (w / 2) << 8 | j.  With m lanes left from lane
 *     pos, the decision stops the word if U_j >= G[m-1]; otherwise lane pos + k is
 *     perturbed for the least k with U_j < G[k], and pos moves to pos + k + 1.
 *     G[k] = floor(2^64 (1 - (1 - P/2^32)^(k+1))): the first-perturbed-lane law
 *     of i.i.d. Bernoulli(P/2^32) lanes, to 2^-64.
 *   Truth tables: function with parents (a_0..a_{k-1}) outputs bit
 *     x = sum_b s[a_b] 2^b of its table.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EPARSE -2
#define ORC_EINVAL -1
#define ORC_ENOMEM -3

enum { DOM_PERT = 1, DOM_SEL = 2, DOM_INIT = 3, DOM_GEO = 4 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from the round function of Salmon et al. (SC'11):  */
/* two 32x32->64 multiplications per round, key bumped by the Weyl constants. */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* One keyed block of the contract. */
static void keyed_block(uint64_t seed, uint64_t traj, uint64_t step, uint32_t domain,
                        uint32_t index, uint32_t out[4]) {
    uint32_t ctr[4], key[2];
    ctr[0] = (uint32_t)(traj & 0xFFFFFFFFu);
    ctr[1] = (uint32_t)(step & 0xFFFFFFFFu);
    ctr[2] = (uint32_t)((step >> 32) & 0xFFFFu) | ((uint32_t)((traj >> 32) & 0xFFFFu) << 16);
    ctr[3] = (domain << 28) | index;
    key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    key[1] = (uint32_t)(seed >> 32);
    orc_philox(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Network model and text parser                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double c;      /* selection probability c_j^{(i)} */
    int k;         /* number of parent nodes */
    int *par;      /* parents a_0..a_{k-1} (original ids) */
    uint8_t *tt;   /* 2^k output bits, one byte each */
} ofun;

typedef struct {
    int nf;
    int cap;
    ofun *f;
} onode;

typedef struct {
    int n;
    double p;
    onode *node;
} onet;

static void net_free(onet *g) {
    if (!g) return;
    if (g->node) {
        for (int i = 0; i < g->n; ++i) {
            for (int j = 0; j < g->node[i].nf; ++j) {
                free(g->node[i].f[j].par);
                free(g->node[i].f[j].tt);
            }
            free(g->node[i].f);
        }
        free(g->node);
    }
    free(g);
}

static int hexval(char ch) {
    if (ch >= '0' && ch <= '9') return ch - '0';
    if (ch >= 'a' && ch <= 'f') return ch - 'a' + 10;
    if (ch >= 'A' && ch <= 'F') return ch - 'A' + 10;
    return -1;
}

/* Text format, one record per line ('#' starts a comment):
 *   pbn <n> <p>
 *   f <node> <c> <k> <a_0> ... <a_{k-1}> <truth table as hex, least significant bit = input 0>
 * The j-th 'f' line of a node is its function f_j.  Numbers may be decimal or
 * C99 hex floats. */
static int parse_net(const char *text, onet **out) {
    onet *g = NULL;
    const char *s = text;
    char *line = NULL;
    size_t linecap = 0;
    int rc = ORC_OK;
    while (*s) {
        const char *e = strchr(s, '\n');
        size_t len = e ? (size_t)(e - s) : strlen(s);
        if (len + 1 > linecap) {
            linecap = len + 1;
            char *nl = (char *)realloc(line, linecap);
            if (!nl) { rc = ORC_ENOMEM; goto done; }
            line = nl;
        }
        memcpy(line, s, len);
        line[len] = 0;
        s = e ? e + 1 : s + len;
        char *hash = strchr(line, '#');
        if (hash) *hash = 0;
        char *save = NULL;
        char *tok = strtok_r(line, " \t\r", &save);
        if (!tok) continue;
        if (strcmp(tok, "pbn") == 0) {
            if (g) { rc = ORC_EPARSE; goto done; }
            char *tn = strtok_r(NULL, " \t\r", &save);
            char *tp = strtok_r(NULL, " \t\r", &save);
            if (!tn || !tp) { rc = ORC_EPARSE; goto done; }
            long n = strtol(tn, NULL, 10);
            double p = strtod(tp, NULL);
            if (n < 1 || n > (1L << 24) || !(p >= 0.0 && p < 1.0)) { rc = ORC_EPARSE; goto done; }
            g = (onet *)calloc(1, sizeof(onet));
            if (!g) { rc = ORC_ENOMEM; goto done; }
            g->n = (int)n;
            g->p = p;
            g->node = (onode *)calloc((size_t)n, sizeof(onode));
            if (!g->node) { rc = ORC_ENOMEM; goto done; }
        } else if (strcmp(tok, "f") == 0) {
            if (!g) { rc = ORC_EPARSE; goto done; }
            char *ti = strtok_r(NULL, " \t\r", &save);
            char *tc = strtok_r(NULL, " \t\r", &save);
            char *tk = strtok_r(NULL, " \t\r", &save);
            if (!ti || !tc || !tk) { rc = ORC_EPARSE; goto done; }
            long i = strtol(ti, NULL, 10);
            double c = strtod(tc, NULL);
            long k = strtol(tk, NULL, 10);
            if (i < 0 || i >= g->n || k < 0 || k > 24 || !(c >= 0.0 && c <= 1.0)) { rc = ORC_EPARSE; goto done; }
            onode *nd = &g->node[i];
            if (nd->nf == nd->cap) {
                int ncap = nd->cap ? 2 * nd->cap : 4;
                ofun *nf = (ofun *)realloc(nd->f, (size_t)ncap * sizeof(ofun));
                if (!nf) { rc = ORC_ENOMEM; goto done; }
                nd->f = nf;
                nd->cap = ncap;
            }
            ofun *f = &nd->f[nd->nf];
            memset(f, 0, sizeof(*f));
            nd->nf++;
            f->c = c;
            f->k = (int)k;
            f->par = (int *)calloc((size_t)(k > 0 ? k : 1), sizeof(int));
            f->tt = (uint8_t *)calloc((size_t)1 << k, 1);
            if (!f->par || !f->tt) { rc = ORC_ENOMEM; goto done; }
            for (long b = 0; b < k; ++b) {
                char *ta = strtok_r(NULL, " \t\r", &save);
                if (!ta) { rc = ORC_EPARSE; goto done; }
                long a = strtol(ta, NULL, 10);
                if (a < 0 || a >= g->n) { rc = ORC_EPARSE; goto done; }
                for (long b2 = 0; b2 < b; ++b2)
                    if (f->par[b2] == a) { rc = ORC_EPARSE; goto done; }
                f->par[b] = (int)a;
            }
            char *th = strtok_r(NULL, " \t\r", &save);
            if (!th) { rc = ORC_EPARSE; goto done; }
            if (th[0] == '0' && (th[1] == 'x' || th[1] == 'X')) th += 2;
            size_t nd_hex = strlen(th);
            size_t nbits = (size_t)1 << k;
            /* walk hex digits from the least significant end */
            for (size_t d = 0; d < nd_hex; ++d) {
                int v = hexval(th[nd_hex - 1 - d]);
                if (v < 0) { rc = ORC_EPARSE; goto done; }
                for (int q = 0; q < 4; ++q) {
                    size_t bit = 4 * d + (size_t)q;
                    int val = (v >> q) & 1;
                    if (bit < nbits) f->tt[bit] = (uint8_t)val;
                    else if (val) { rc = ORC_EPARSE; goto done; }
                }
            }
            if (strtok_r(NULL, " \t\r", &save)) { rc = ORC_EPARSE; goto done; }
        } else {
            rc = ORC_EPARSE;
            goto done;
        }
    }
    if (!g) { rc = ORC_EPARSE; goto done; }
    for (int i = 0; i < g->n; ++i) {
        if (g->node[i].nf < 1) { rc = ORC_EPARSE; goto done; }
        double sum = 0.0;
        for (int j = 0; j < g->node[i].nf; ++j) sum += g->node[i].f[j].c;
        if (fabs(sum - 1.0) > 1e-9) { rc = ORC_EPARSE; goto done; }
    }
done:
    free(line);
    if (rc != ORC_OK) { net_free(g); g = NULL; }
    *out = g;
    return rc;
}

/* Perturbation threshold P = floor(p * 2^32): p * 2^32 is exact in fp64. */
static uint64_t pert_threshold(double p) { return (uint64_t)floor(p * 4294967296.0); }

/* Selection thresholds T_1..T_{l-1} of a node (T_0 = 0, T_l = 2^32 implied). */
static void sel_thresholds(const onode *nd, uint64_t *T) {
    double C = 0.0;
    for (int j = 1; j < nd->nf; ++j) {
        C = C + nd->f[j - 1].c;
        double v = floor(C * 4294967296.0);
        T[j] = v >= 4294967296.0 ? (uint64_t)1 << 32 : (uint64_t)v;
    }
}

/* Thresholds of the geometric sampler, G[k] = floor(2^64 (1 - (1 - P/2^32)^(k+1)))
 * for k = 0..63, in exact integer arithmetic: with a = 2^32 - P,
 * (1 - P/2^32)^(k+1) = a^(k+1) / 2^(32(k+1)), so
 * G[k] = 2^64 - ceil(a^(k+1) / 2^(32(k+1) - 64)).  a^(k+1) is kept as
 * little-endian 32-bit limbs. */
static void geo_thresholds(uint64_t P, uint64_t G[64]) {
    if (P == 0) {
        for (int k = 0; k < 64; ++k) G[k] = 0;
        return;
    }
    const uint64_t a = ((uint64_t)1 << 32) - P; /* 1 <= a < 2^32 */
    uint32_t limb[70];
    int nl = 1;
    limb[0] = 1;
    for (int k = 0; k < 64; ++k) {
        /* limb <- limb * a */
        uint64_t carry = 0;
        for (int i = 0; i < nl; ++i) {
            uint64_t v = (uint64_t)limb[i] * a + carry;
            limb[i] = (uint32_t)v;
            carry = v >> 32;
        }
        if (carry) limb[nl++] = (uint32_t)carry;
        /* q = ceil(a^(k+1) / 2^(32(k+1) - 64)) */
        uint64_t q;
        if (k == 0) {
            q = a << 32; /* exact: the divisor is 2^-32 */
        } else {
            const int drop = k - 1; /* limbs shifted out */
            uint64_t lo = drop < nl ? limb[drop] : 0, hi = drop + 1 < nl ? limb[drop + 1] : 0;
            q = (hi << 32) | lo;
            int rest = 0;
            for (int i = 0; i < drop && i < nl; ++i) rest |= limb[i] != 0;
            q += (uint64_t)rest;
        }
        G[k] = (uint64_t)0 - q; /* 2^64 - q, q >= 1 */
    }
}

/* Per-network data the simulator needs besides the model itself. */
typedef struct {
    const onet *g;
    uint64_t P;
    int *rank;        /* rank among nodes with >= 2 functions, or -1 */
    uint64_t *thr;    /* thr[i * 16 + j] = T_j of node i (j < 16) */
    uint64_t G[64];   /* thresholds of the geometric sampler */
    int sampler;      /* 0: bit-sliced levels (PERT), 1: geometric (GEO) */
} octx;

static int ctx_init(octx *cx, const onet *g) {
    cx->g = g;
    cx->P = pert_threshold(g->p);
    geo_thresholds(cx->P, cx->G);
    cx->rank = (int *)malloc((size_t)g->n * sizeof(int));
    cx->thr = (uint64_t *)calloc((size_t)g->n * 16, sizeof(uint64_t));
    if (!cx->rank || !cx->thr) return ORC_ENOMEM;
    int r = 0;
    for (int i = 0; i < g->n; ++i) {
        if (g->node[i].nf > 16) return ORC_EINVAL;
        cx->rank[i] = g->node[i].nf >= 2 ? r++ : -1;
        sel_thresholds(&g->node[i], cx->thr + (size_t)i * 16);
    }
    return ORC_OK;
}

static void ctx_free(octx *cx) {
    free(cx->rank);
    free(cx->thr);
}

/* gamma_i for all nodes of one (trajectory, step): the plain definition,
 * all 32 levels assembled into u_i and compared with P. */
static int draw_geo(const octx *cx, uint64_t seed, uint64_t traj, uint64_t step, uint8_t *gamma);

static int draw_pert(const octx *cx, uint64_t seed, uint64_t traj, uint64_t step, uint8_t *gamma) {
    if (cx->sampler == 1) return draw_geo(cx, seed, traj, step, gamma);
    int n = cx->g->n;
    int W = (n + 63) / 64;
    int any = 0;
    for (int w = 0; w < W; ++w) {
        uint64_t level[32];
        for (int h = 0; h < 16; ++h) {
            uint32_t x[4];
            keyed_block(seed, traj, step, DOM_PERT, ((uint32_t)w << 4) | (uint32_t)h, x);
            level[2 * h] = ((uint64_t)x[1] << 32) | x[0];
            level[2 * h + 1] = ((uint64_t)x[3] << 32) | x[2];
        }
        for (int b = 0; b < 64; ++b) {
            int i = 64 * w + b;
            if (i >= n) break;
            uint64_t u = 0;
            for (int l = 0; l < 32; ++l) u |= ((level[l] >> b) & 1u) << (31 - l);
            gamma[i] = (uint8_t)(u < cx->P);
            any |= gamma[i];
        }
    }
    return any;
}

/* gamma_i of the geometric sampler (GEO): per word, the first perturbed lane among
 * the remaining ones is drawn by inverting its distribution with one 64-bit
 * uniform, until a uniform says that none of the remaining lanes is perturbed. */
static int draw_geo(const octx *cx, uint64_t seed, uint64_t traj, uint64_t step, uint8_t *gamma) {
    int n = cx->g->n;
    int W = (n + 63) / 64;
    int any = 0;
    for (int i = 0; i < n; ++i) gamma[i] = 0;
    for (int w = 0; w < W; ++w) {
        int L = n - 64 * w < 64 ? n - 64 * w : 64;
        int pos = 0;
        uint32_t j = 0;
        while (pos < L) {
            int m = L - pos;
            uint32_t x[4];
            keyed_block(seed, traj, step, DOM_GEO, ((uint32_t)(w / 2) << 8) | j, x);
            uint64_t U = (w % 2 == 0) ? (((uint64_t)x[1] << 32) | x[0]) : (((uint64_t)x[3] << 32) | x[2]);
            ++j;
            if (U >= cx->G[m - 1]) break;
            int k = 0;
            while (U >= cx->G[k]) ++k;
            gamma[64 * w + pos + k] = 1;
            any = 1;
            pos += k + 1;
        }
    }
    return any;
}

/* 0-based function choice of every node for one (trajectory, step). */
static void draw_sel(const octx *cx, uint64_t seed, uint64_t traj, uint64_t step, uint8_t *choice) {
    const onet *g = cx->g;
    for (int i = 0; i < g->n; ++i) {
        int r = cx->rank[i];
        if (r < 0) { choice[i] = 0; continue; }
        uint32_t x[4];
        keyed_block(seed, traj, step, DOM_SEL, (uint32_t)r >> 2, x);
        uint64_t u = x[r & 3];
        int j = 0;
        for (int t = 1; t < g->node[i].nf; ++t)
            if (u >= cx->thr[(size_t)i * 16 + t]) ++j;
        choice[i] = (uint8_t)j;
    }
}

static void draw_init(const octx *cx, uint64_t seed, uint64_t traj, uint8_t *s) {
    int n = cx->g->n;
    for (int i = 0; i < n; ++i) {
        int w = i / 64, b = i % 64;
        uint32_t x[4];
        keyed_block(seed, traj, 0, DOM_INIT, (uint32_t)w >> 1, x);
        uint64_t word = (w % 2 == 0) ? (((uint64_t)x[1] << 32) | x[0]) : (((uint64_t)x[3] << 32) | x[2]);
        s[i] = (uint8_t)((word >> b) & 1u);
    }
}

static int eval_fun(const ofun *f, const uint8_t *s) {
    uint64_t x = 0;
    for (int b = 0; b < f->k; ++b) x |= (uint64_t)s[f->par[b]] << b;
    return f->tt[x];
}

/* ------------------------------------------------------------------------ */
/* Simulation                                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    const octx *cx;
    uint64_t seed, traj_begin, step_begin, n_steps, count_from;
    const int32_t *meta_ids;
    const uint8_t *meta_vals;
    int n_meta;
    const uint8_t *init_states;
    uint8_t *final_states;
    uint64_t *counts;
    uint8_t *trace;
    uint64_t t_lo, t_hi; /* local trajectory range of this worker */
    int per_node;        /* 0: Eq. 1; 1: node-wise flips */
    int rc;
} sim_job;

static int meta_hit(const sim_job *jb, const uint8_t *s) {
    for (int m = 0; m < jb->n_meta; ++m)
        if (s[jb->meta_ids[m]] != jb->meta_vals[m]) return 0;
    return 1;
}

static void *sim_worker(void *arg) {
    sim_job *jb = (sim_job *)arg;
    const octx *cx = jb->cx;
    const onet *g = cx->g;
    int n = g->n;
    uint8_t *s = (uint8_t *)malloc((size_t)n);
    uint8_t *s2 = (uint8_t *)malloc((size_t)n);
    uint8_t *gam = (uint8_t *)malloc((size_t)n);
    uint8_t *ch = (uint8_t *)malloc((size_t)n);
    if (!s || !s2 || !gam || !ch) { jb->rc = ORC_ENOMEM; goto out; }
    for (uint64_t lt = jb->t_lo; lt < jb->t_hi; ++lt) {
        uint64_t traj = jb->traj_begin + lt;
        if (jb->init_states) memcpy(s, jb->init_states + lt * (uint64_t)n, (size_t)n);
        else draw_init(cx, jb->seed, traj, s);
        uint64_t cnt[5] = {0, 0, 0, 0, 0}; /* V, n00, n01, n10, n11 */
        int z_prev = meta_hit(jb, s);
        /* the initial state belongs to the window only when this run starts the
         * trajectory (keyed s(0)); a run from given states continues one whose
         * earlier run produced, and counted, that state */
        if (!jb->init_states && jb->step_begin >= jb->count_from) cnt[0] += (uint64_t)z_prev;
        for (uint64_t k = 0; k < jb->n_steps; ++k) {
            uint64_t t = jb->step_begin + k;
            /* Eq. 1: perturb if any gamma_i is set, else apply selected functions. */
            if (jb->per_node) {
                /* node-wise: a flipped node negates, every other node applies its
                 * selected function to the old state */
                draw_pert(cx, jb->seed, traj, t, gam);
                draw_sel(cx, jb->seed, traj, t, ch);
                for (int i = 0; i < n; ++i)
                    s2[i] = gam[i] ? (uint8_t)(s[i] ^ 1u) : (uint8_t)eval_fun(&g->node[i].f[ch[i]], s);
                memcpy(s, s2, (size_t)n);
            } else if (draw_pert(cx, jb->seed, traj, t, gam)) {
                for (int i = 0; i < n; ++i) s[i] ^= gam[i];
            } else {
                draw_sel(cx, jb->seed, traj, t, ch);
                for (int i = 0; i < n; ++i) s2[i] = (uint8_t)eval_fun(&g->node[i].f[ch[i]], s);
                memcpy(s, s2, (size_t)n);
            }
            int z = meta_hit(jb, s);
            if (t + 1 >= jb->count_from) cnt[0] += (uint64_t)z;
            if (t >= jb->count_from) cnt[1 + 2 * z_prev + z] += 1;
            z_prev = z;
            if (jb->trace) memcpy(jb->trace + (lt * jb->n_steps + k) * (uint64_t)n, s, (size_t)n);
        }
        if (jb->final_states) memcpy(jb->final_states + lt * (uint64_t)n, s, (size_t)n);
        if (jb->counts) memcpy(jb->counts + lt * 5, cnt, sizeof(cnt));
    }
out:
    free(s); free(s2); free(gam); free(ch);
    return NULL;
}

/* Simulate n_traj trajectories (ids traj_begin ...) for steps
 * step_begin .. step_begin + n_steps - 1.  init_states (n_traj x n bytes) or
 * NULL for the keyed initial state (then step_begin must be 0).  counts gets
 * [V, n00, n01, n10, n11] per trajectory over states with index >= count_from:
 * the states the run produces, the pairs it steps through, and its initial state
 * only when the run starts the trajectory (keyed), so that runs resumed from saved
 * states add up to one run over all the steps (Sec. 4.2's chain, cut anywhere).
 * trace (optional) gets the state after every step: n_traj x n_steps x n. */
int orc_simulate_ex(const char *text, uint64_t seed, uint64_t traj_begin, uint64_t n_traj,
                    uint64_t step_begin, uint64_t n_steps, uint64_t count_from,
                    const int32_t *meta_ids, const uint8_t *meta_vals, int n_meta,
                    const uint8_t *init_states, uint8_t *final_states, uint64_t *counts,
                    uint8_t *trace, int nthreads, int semantics, int sampler);

int orc_simulate(const char *text, uint64_t seed, uint64_t traj_begin, uint64_t n_traj,
                 uint64_t step_begin, uint64_t n_steps, uint64_t count_from,
                 const int32_t *meta_ids, const uint8_t *meta_vals, int n_meta,
                 const uint8_t *init_states, uint8_t *final_states, uint64_t *counts,
                 uint8_t *trace, int nthreads) {
    return orc_simulate_ex(text, seed, traj_begin, n_traj, step_begin, n_steps, count_from, meta_ids,
                           meta_vals, n_meta, init_states, final_states, counts, trace, nthreads, 0, 0);
}

/* As orc_simulate; semantics 0 = Eq. 1, 1 = node-wise flips. */
int orc_simulate_sem(const char *text, uint64_t seed, uint64_t traj_begin, uint64_t n_traj,
                     uint64_t step_begin, uint64_t n_steps, uint64_t count_from,
                     const int32_t *meta_ids, const uint8_t *meta_vals, int n_meta,
                     const uint8_t *init_states, uint8_t *final_states, uint64_t *counts,
                     uint8_t *trace, int nthreads, int semantics) {
    return orc_simulate_ex(text, seed, traj_begin, n_traj, step_begin, n_steps, count_from, meta_ids,
                           meta_vals, n_meta, init_states, final_states, counts, trace, nthreads, semantics, 0);
}

/* As orc_simulate_sem; sampler 0 = bit-sliced levels (PERT), 1 = geometric (GEO). */
int orc_simulate_ex(const char *text, uint64_t seed, uint64_t traj_begin, uint64_t n_traj,
                    uint64_t step_begin, uint64_t n_steps, uint64_t count_from,
                    const int32_t *meta_ids, const uint8_t *meta_vals, int n_meta,
                    const uint8_t *init_states, uint8_t *final_states, uint64_t *counts,
                    uint8_t *trace, int nthreads, int semantics, int sampler) {
    if (semantics != 0 && semantics != 1) return ORC_EINVAL;
    if (sampler != 0 && sampler != 1) return ORC_EINVAL;
    onet *g = NULL;
    int rc = parse_net(text, &g);
    if (rc) return rc;
    if (!init_states && step_begin != 0) { net_free(g); return ORC_EINVAL; }
    for (int m = 0; m < n_meta; ++m)
        if (meta_ids[m] < 0 || meta_ids[m] >= g->n) { net_free(g); return ORC_EINVAL; }
    octx cx;
    memset(&cx, 0, sizeof(cx));
    rc = ctx_init(&cx, g);
    if (rc) { ctx_free(&cx); net_free(g); return rc; }
    cx.sampler = sampler;
    if (nthreads < 1) nthreads = 1;
    if ((uint64_t)nthreads > n_traj) nthreads = n_traj > 0 ? (int)n_traj : 1;
    sim_job *jobs = (sim_job *)calloc((size_t)nthreads, sizeof(sim_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); ctx_free(&cx); net_free(g); return ORC_ENOMEM; }
    for (int w = 0; w < nthreads; ++w) {
        sim_job *jb = &jobs[w];
        jb->cx = &cx; jb->seed = seed; jb->traj_begin = traj_begin;
        jb->step_begin = step_begin; jb->n_steps = n_steps; jb->count_from = count_from;
        jb->meta_ids = meta_ids; jb->meta_vals = meta_vals; jb->n_meta = n_meta;
        jb->init_states = init_states; jb->final_states = final_states;
        jb->counts = counts; jb->trace = trace;
        jb->per_node = semantics;
        jb->t_lo = n_traj * (uint64_t)w / (uint64_t)nthreads;
        jb->t_hi = n_traj * (uint64_t)(w + 1) / (uint64_t)nthreads;
    }
    if (nthreads == 1) {
        sim_worker(&jobs[0]);
    } else {
        for (int w = 0; w < nthreads; ++w) pthread_create(&th[w], NULL, sim_worker, &jobs[w]);
        for (int w = 0; w < nthreads; ++w) pthread_join(th[w], NULL);
    }
    for (int w = 0; w < nthreads; ++w) if (jobs[w].rc) rc = jobs[w].rc;
    free(jobs); free(th);
    ctx_free(&cx);
    net_free(g);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Draw inspection (for pins)                                                */
/* ------------------------------------------------------------------------ */
int orc_draws(const char *text, uint64_t seed, uint64_t traj, uint64_t step,
              uint8_t *gamma, uint8_t *choice, uint8_t *init, int *any) {
    onet *g = NULL;
    int rc = parse_net(text, &g);
    if (rc) return rc;
    octx cx;
    memset(&cx, 0, sizeof(cx));
    rc = ctx_init(&cx, g);
    if (!rc) {
        int a = draw_pert(&cx, seed, traj, step, gamma);
        if (any) *any = a;
        draw_sel(&cx, seed, traj, step, choice);
        draw_init(&cx, seed, traj, init);
    }
    ctx_free(&cx);
    net_free(g);
    return rc;
}

/* The keyed draws of one (trajectory, step) under a given perturbation sampler. */
int orc_draws_ex(const char *text, uint64_t seed, uint64_t traj, uint64_t step, int sampler,
                 uint8_t *gamma, int *any) {
    onet *g = NULL;
    int rc = parse_net(text, &g);
    if (rc) return rc;
    octx cx;
    memset(&cx, 0, sizeof(cx));
    rc = ctx_init(&cx, g);
    if (!rc) {
        cx.sampler = sampler;
        int a = draw_pert(&cx, seed, traj, step, gamma);
        if (any) *any = a;
    }
    ctx_free(&cx);
    net_free(g);
    return rc;
}

/* The geometric sampler's thresholds G[0..63] for perturbation rate p. */
void orc_geo_thresholds(double p, uint64_t *G) { geo_thresholds(pert_threshold(p), G); }

/* Integer thresholds of node i: P, then T_1..T_{l-1}.  Returns l. */
int orc_thresholds(const char *text, int node, uint64_t *P, uint64_t *T) {
    onet *g = NULL;
    int rc = parse_net(text, &g);
    if (rc) return rc;
    if (node < 0 || node >= g->n || g->node[node].nf > 16) { net_free(g); return ORC_EINVAL; }
    *P = pert_threshold(g->p);
    uint64_t t[16] = {0};
    sel_thresholds(&g->node[node], t);
    int l = g->node[node].nf;
    for (int j = 1; j < l; ++j) T[j - 1] = t[j];
    net_free(g);
    return l;
}

/* Network shape: n, number of functions, sum of parents (density numerator). */
int orc_shape(const char *text, int *n, int *n_fun, long *sum_parents, double *p) {
    onet *g = NULL;
    int rc = parse_net(text, &g);
    if (rc) return rc;
    *n = g->n;
    *p = g->p;
    int nf = 0;
    long sp = 0;
    for (int i = 0; i < g->n; ++i) {
        nf += g->node[i].nf;
        for (int j = 0; j < g->node[i].nf; ++j) sp += g->node[i].f[j].k;
    }
    *n_fun = nf;
    *sum_parents = sp;
    net_free(g);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Exact transition matrix of the perturbed PBN (Eq. 1) for n <= 14.          */
/* With p' = P / 2^32 and c'_j = (T_j - T_{j-1}) / 2^32 (the probabilities     */
/* the integer thresholds realise):                                           */
/*   Pr(s -> s') = [s' != s] p'^h (1-p')^(n-h)   (h = Hamming distance)       */
/*              + (1-p')^n prod_i q_i(s, s'_i),  q_i(s,1) = sum_j c'_j f_j(s) */
/* States are indexed by sum_i s_i 2^i.  M is row-major, 2^n x 2^n.           */
/* ------------------------------------------------------------------------ */
int orc_transition_matrix_sem(const char *text, int semantics, double *M);

int orc_transition_matrix(const char *text, double *M) { return orc_transition_matrix_sem(text, 0, M); }

/* Node-wise variant (semantics 1): the nodes move independently given s,
 *   Pr(s -> s') = prod_i [ p' [s'_i != s_i] + (1-p') q_i(s, s'_i) ]. */
int orc_transition_matrix_sem(const char *text, int semantics, double *M) {
    if (semantics != 0 && semantics != 1) return ORC_EINVAL;
    onet *g = NULL;
    int rc = parse_net(text, &g);
    if (rc) return rc;
    int n = g->n;
    if (n > 14) { net_free(g); return ORC_EINVAL; }
    octx cx;
    memset(&cx, 0, sizeof(cx));
    rc = ctx_init(&cx, g);
    if (rc) { ctx_free(&cx); net_free(g); return rc; }
    size_t S = (size_t)1 << n;
    double pe = (double)cx.P / 4294967296.0;
    double *pw = (double *)malloc((size_t)(n + 1) * sizeof(double));
    double *q1 = (double *)malloc((size_t)n * sizeof(double));
    double *row = (double *)malloc(S * sizeof(double));
    uint8_t *st = (uint8_t *)malloc((size_t)n);
    if (!pw || !q1 || !row || !st) { rc = ORC_ENOMEM; goto out; }
    /* pw[h] = p'^h (1-p')^(n-h) */
    for (int h = 0; h <= n; ++h) {
        double v = 1.0;
        for (int a = 0; a < h; ++a) v *= pe;
        for (int a = 0; a < n - h; ++a) v *= (1.0 - pe);
        pw[h] = v;
    }
    for (size_t s = 0; s < S; ++s) {
        for (int i = 0; i < n; ++i) st[i] = (uint8_t)((s >> i) & 1u);
        for (int i = 0; i < n; ++i) {
            const onode *nd = &g->node[i];
            const uint64_t *T = cx.thr + (size_t)i * 16;
            double q = 0.0;
            for (int j = 0; j < nd->nf; ++j) {
                uint64_t lo = j == 0 ? 0 : T[j];
                uint64_t hi = j == nd->nf - 1 ? ((uint64_t)1 << 32) : T[j + 1];
                double cj = hi > lo ? (double)(hi - lo) / 4294967296.0 : 0.0;
                if (eval_fun(&nd->f[j], st)) q += cj;
            }
            q1[i] = q;
        }
        if (semantics == 1) {
            /* node i is 1 next with probability p' [s_i = 0] + (1-p') q_i(s, 1) */
            for (int i = 0; i < n; ++i) q1[i] = pe * (double)(st[i] ^ 1u) + (1.0 - pe) * q1[i];
        }
        /* product distribution over s' built one node at a time */
        row[0] = semantics == 1 ? 1.0 : pw[0];
        size_t len = 1;
        for (int i = 0; i < n; ++i) {
            for (size_t a = 0; a < len; ++a) {
                double v = row[a];
                row[a] = v * (1.0 - q1[i]);
                row[a + len] = v * q1[i];
            }
            len <<= 1;
        }
        for (size_t s2 = 0; s2 < S; ++s2) {
            if (semantics == 0 && s2 != s) row[s2] += pw[__builtin_popcountll((unsigned long long)(s ^ s2))];
            M[s * S + s2] = row[s2];
        }
    }
out:
    free(pw); free(q1); free(row); free(st);
    ctx_free(&cx);
    net_free(g);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Definition 1 (leaf node), taken literally: a node is a leaf iff it is not */
/* of interest and every child it has (self-edges not counted) is a leaf;     */
/* iterate until nothing changes.  Children are structural: u is a child of   */
/* v iff v is a parent of some function of u.                                 */
/* ------------------------------------------------------------------------ */
int orc_leaves(const char *text, const int32_t *interest, int n_interest, uint8_t *is_leaf) {
    onet *g = NULL;
    int rc = parse_net(text, &g);
    if (rc) return rc;
    int n = g->n;
    uint8_t *intr = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *child = (uint8_t *)calloc((size_t)n * (size_t)n, 1); /* child[v*n+u] */
    if (!intr || !child) { free(intr); free(child); net_free(g); return ORC_ENOMEM; }
    for (int m = 0; m < n_interest; ++m) {
        if (interest[m] < 0 || interest[m] >= n) { free(intr); free(child); net_free(g); return ORC_EINVAL; }
        intr[interest[m]] = 1;
    }
    for (int u = 0; u < n; ++u)
        for (int j = 0; j < g->node[u].nf; ++j)
            for (int b = 0; b < g->node[u].f[j].k; ++b) {
                int v = g->node[u].f[j].par[b];
                if (v != u) child[(size_t)v * n + u] = 1;
            }
    memset(is_leaf, 0, (size_t)n);
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int v = 0; v < n; ++v) {
            if (is_leaf[v] || intr[v]) continue;
            int ok = 1;
            for (int u = 0; u < n && ok; ++u)
                if (child[(size_t)v * n + u] && !is_leaf[u]) ok = 0;
            if (ok) { is_leaf[v] = 1; changed = 1; }
        }
    }
    free(intr); free(child);
    net_free(g);
    return ORC_OK;
}


/* Reachability variant of the reduction: node v is kept iff it is a node of
 * interest or one of its children (self-edges ignored) is kept, iterated to the
 * fixed point, i.e. iff some node of interest can be reached from v along
 * parent -> child edges.  removed[v] = 1 for the other nodes. */
int orc_reach(const char *text, const int32_t *interest, int n_interest, uint8_t *removed) {
    onet *g = NULL;
    int rc = parse_net(text, &g);
    if (rc) return rc;
    int n = g->n;
    uint8_t *keep = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *child = (uint8_t *)calloc((size_t)n * (size_t)n, 1); /* child[v*n+u] */
    if (!keep || !child) { free(keep); free(child); net_free(g); return ORC_ENOMEM; }
    for (int m = 0; m < n_interest; ++m) {
        if (interest[m] < 0 || interest[m] >= n) { free(keep); free(child); net_free(g); return ORC_EINVAL; }
        keep[interest[m]] = 1;
    }
    for (int u = 0; u < n; ++u)
        for (int j = 0; j < g->node[u].nf; ++j)
            for (int b = 0; b < g->node[u].f[j].k; ++b) {
                int v = g->node[u].f[j].par[b];
                if (v != u) child[(size_t)v * n + u] = 1;
            }
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int v = 0; v < n; ++v) {
            if (keep[v]) continue;
            for (int u = 0; u < n; ++u)
                if (child[(size_t)v * n + u] && keep[u]) { keep[v] = 1; changed = 1; break; }
        }
    }
    for (int v = 0; v < n; ++v) removed[v] = (uint8_t)!keep[v];
    free(keep); free(child);
    net_free(g);
    return ORC_OK;
}
