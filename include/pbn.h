/*
 * pbn.h -- C ABI of the GB300-native probabilistic Boolean network simulator.
 *
 * The library implements the structure-based simulation of Mizera, Pang and Yuan,
 * "Fast Simulation of Probabilistic Boolean Networks": leaf-node reduction
 * (Sec. 3.1, Definition 1), node grouping into merged predictor functions
 * (Sec. 3.3, Eq. 2, Algorithms 3-4) and the per-step simulation of Algorithm 5,
 * run for many trajectories at once by CUDA kernels for sm_103a.  Every step
 * follows Eq. 1 (Sec. 2.1): each node is flipped with probability p; if any node
 * flipped, the next state is s XOR gamma, otherwise every node applies a predictor
 * function drawn from its selection probabilities.  The kernels also count the
 * visits and transitions of a meta-state that the two-state Markov chain
 * estimator (Sec. 4.2) consumes.
 *
 * Random draws are keyed: draw = Philox4x32-10(key = seed, counter = (trajectory,
 * step, domain, index)) with indices defined on ORIGINAL node ids, so results do
 * not depend on launch shape, reduction or grouping.  Domains:
 *   PERT (1): node i = 64w + b, index w << 4 | h gives levels 2h (x1:x0) and
 *             2h+1 (x3:x2); u_i has bit 31-l equal to bit b of level l, and node i
 *             is perturbed iff u_i < P = floor(p * 2^32).
 *   SEL  (2): nodes with >= 2 functions ranked by ascending id; rank r reads word
 *             x_{r mod 4} of index r / 4; the 0-based choice is the number of
 *             thresholds T_j = min(floor(C_j 2^32), 2^32), C_j = c_1 + ... + c_j
 *             summed left to right in fp64, j = 1..l-1, with u >= T_j.
 *   INIT (3): step 0; word w of s(0) is x1:x0 (w even) or x3:x2 (w odd) of
 *             index w / 2.
 * Counter: c0 = trajectory bits 0..31, c1 = step bits 0..31,
 * c2 = step bits 32..47 | trajectory bits 32..47 << 16, c3 = domain << 28 | index.
 *
 * Conventions.
 *  - Every function returns a pbn status (0 = PBN_OK, negative = error).  No C++
 *    exception crosses this boundary.  pbn_last_error_detail() gives a message
 *    for the calling thread's last error.
 *  - pbn_net and pbn_plan are opaque, created by the library, freed with the
 *    matching *_free call, and immutable after creation: concurrent
 *    pbn_simulate calls on one plan are safe.
 *  - Device buffers are owned by the caller and passed as raw device pointers
 *    together with a cudaStream_t (as void*).  The library allocates no device
 *    memory and never synchronises the caller's stream.
 */
#ifndef PBN_H
#define PBN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define PBN_OK 0
#define PBN_EINVAL (-1)   /* an argument is out of range or inconsistent */
#define PBN_EPARSE (-2)   /* the network text is malformed */
#define PBN_ENOMEM (-3)   /* host allocation failed */
#define PBN_ECUDA (-4)    /* a CUDA runtime call or kernel launch failed */
#define PBN_ETOOBIG (-5)  /* a plan does not fit the device limits (tables, shared memory) */
#define PBN_ETIMEOUT (-6) /* a bounded device wait gave up (see PBN_DEV_* bits) */
#define PBN_EDEVICE (-7)  /* a kernel reported an error in its status word */

/* Bits a kernel ORs into the caller's device status word. */
#define PBN_DEV_STAGE_TIMEOUT 0x1u /* the bulk copy of plan tables into shared memory did not complete in time */
#define PBN_DEV_BAD_PLAN 0x2u      /* the device image does not carry the expected header */
#define PBN_DEV_BAD_MODULE 0x4u    /* a compiled batch's linked parts disagree on the kernel's shared
                                      memory; the work item was skipped */

/* ---- networks ---------------------------------------------------------------- */
typedef struct pbn_net pbn_net;
typedef struct pbn_plan pbn_plan;

/* Parse a PBN G(X, F) with perturbation rate p (Sec. 2.1) from text:
 *     pbn <n> <p>
 *     f <node> <c> <k> <a_0> ... <a_{k-1}> <truth table hex>
 * one 'f' line per predictor function f_j of node <node> (in order j = 1, 2, ...),
 * with selection probability c, k distinct parents and a truth table whose bit
 * x = sum_b s[a_b] 2^b is the output.  Numbers may be decimal or C99 hex floats.
 * Requires 1 <= n <= 2^24, 0 <= p < 1, k <= 24, 1..16 functions per node, c >= 0
 * and |sum_j c_j - 1| <= 1e-9 per node.  text need not be NUL-terminated.
 * On success *out owns a new network (free with pbn_net_free).
 * Errors: PBN_EINVAL (NULL argument), PBN_EPARSE (malformed text), PBN_ENOMEM. */
int pbn_load(const char* text, size_t len, pbn_net** out);

/* The same network from arrays (Sec. 2.1: node set, predictor functions with
 * their selection probabilities, perturbation rate p).  Function f (0 <= f <
 * n_functions) belongs to node fun_node[f]; the functions of one node are its
 * f_1, f_2, ... in the order they appear.  Its fun_k[f] parents follow those of
 * function f - 1 in `parents`, and its truth table takes the next ceil(2^k / 64)
 * 64-bit words of `tt`: bit x (least significant first) is the output on the input
 * pattern x = sum_b s[a_b] 2^b, and bits at x >= 2^k must be 0.  The arrays are
 * host memory, read during the call only.  Same requirements as pbn_load.
 * On success *out owns a new network (free with pbn_net_free).
 * Errors: PBN_EINVAL (NULL argument or a requirement not met), PBN_ENOMEM. */
typedef struct {
    uint32_t n;                /* nodes */
    uint32_t n_functions;      /* predictor functions of all nodes */
    double p;                  /* perturbation rate */
    const uint32_t* fun_node;  /* [n_functions] node of each function */
    const double* fun_c;       /* [n_functions] selection probability c */
    const uint32_t* fun_k;     /* [n_functions] number of parents, <= 24 */
    const uint32_t* parents;   /* [sum fun_k] ordered distinct parents, function by function */
    const uint64_t* tt;        /* [sum ceil(2^k / 64)] truth tables, function by function */
} pbn_net_desc;

int pbn_load_arrays(const pbn_net_desc* desc, pbn_net** out);

typedef struct {
    uint32_t n;            /* nodes of the original network */
    uint32_t n_retained;   /* nodes kept by pbn_reduce (n for an unreduced network) */
    uint32_t n_functions;  /* N_F, total number of predictor functions */
    uint32_t n_multi;      /* nodes with >= 2 predictor functions (SEL ranks) */
    double p;              /* perturbation rate as given */
    uint64_t P;            /* floor(p * 2^32): node perturbed iff its u < P */
    double density;        /* D(G) = (1/n) sum_i phi(i), Sec. 2.1 */
} pbn_net_info;

/* Shape of a network.  Errors: PBN_EINVAL. */
int pbn_net_info_get(const pbn_net* net, pbn_net_info* out);

/* Leaf-node reduction (Sec. 3.1, Definition 1).  A node is a leaf iff it is not
 * in interest[] and each of its children (nodes having it as a parent of some
 * function; self-edges not counted) is a leaf, applied until nothing changes.
 * *reduced is a new network that keeps every node of net (leaves still take part
 * in the perturbation draw, Sec. 3.1) but marks only the retained nodes for
 * simulation.  retained_ids (capacity net's n, may be NULL) receives the retained
 * original ids in ascending order and *n_retained their number (may be NULL).
 * The nodes of interest are the meta-state nodes of the analysis; they are always
 * retained.  Errors: PBN_EINVAL (NULL net/reduced, interest id out of range),
 * PBN_ENOMEM. */
int pbn_reduce(const pbn_net* net, const uint32_t* interest, uint32_t n_interest,
               pbn_net** reduced, uint32_t* retained_ids, uint32_t* n_retained);

/* pbn_reduce with a choice of rule.  PBN_REDUCE_LEAVES is Definition 1 (the rule
 * of pbn_reduce).  PBN_REDUCE_REACH retains exactly the nodes from which a node of
 * interest can be reached along parent -> child edges (the nodes of interest
 * included): a node that reaches none cannot influence them, so their
 * trajectories are unchanged (the same argument as Sec. 3.1's for leaves).  It
 * also removes cycles of such nodes, which Definition 1 keeps; its retained set is
 * a subset of Definition 1's.  Errors: as pbn_reduce, and PBN_EINVAL for an
 * unknown rule. */
#define PBN_REDUCE_LEAVES 0u
#define PBN_REDUCE_REACH 1u
int pbn_reduce_rule(const pbn_net* net, const uint32_t* interest, uint32_t n_interest, uint32_t rule,
                    pbn_net** reduced, uint32_t* retained_ids, uint32_t* n_retained);

/* ---- plans ------------------------------------------------------------------- */
#define PBN_PLAN_GROUPED 0u /* node grouping of Sec. 3.3 (Eq. 2, Algorithms 3-4) */
#define PBN_PLAN_PLAIN 1u   /* one node per group: the unmerged per-node method */

/* Perturbation semantics of a plan.  PBN_SEM_EQ1 is Eq. 1: if any node (leaves
 * included) is perturbed, s(t+1) = s(t) XOR gamma and no function is applied.
 * PBN_SEM_NODEWISE is the node-by-node reading of Sec. 2.1's description: a
 * perturbed node takes NOT s_i, every other node applies its selected function
 * to s(t), in every step.  Both consume the same keyed draws. */
#define PBN_SEM_EQ1 0u
#define PBN_SEM_NODEWISE 1u

/* Perturbation sampler of a plan (both give i.i.d. Bernoulli(p') lanes, p' = P/2^32,
 * from different keyed draws, so their trajectories differ).
 * PBN_PERT_BITSLICED is the keyed contract's PERT domain: bit-sliced comparison of
 * every lane's 32-bit uniform with P, level by level (a 64-lane word needs about
 * 4 Philox blocks per step).
 * PBN_PERT_GEOMETRIC draws, per 64-node word, the first perturbed lane among the
 * remaining ones by inverting its distribution with one 64-bit uniform (GEO domain,
 * index (w / 2) << 8 | j, x1:x0 for even w, x3:x2 for odd w), against the
 * thresholds G[k] = floor(2^64 (1 - (1 - p')^(k+1))) computed in exact integer
 * arithmetic: with m lanes left from lane pos, U >= G[m-1] ends the word, else lane
 * pos + k is perturbed for the least k with U < G[k].  One Philox block decides two
 * words in the common case; the law equals the bit-sliced one to 2^-64. */
#define PBN_PERT_BITSLICED 0u
#define PBN_PERT_GEOMETRIC 1u

typedef struct {
    uint32_t mode;          /* PBN_PLAN_GROUPED or PBN_PLAN_PLAIN */
    uint32_t max_inputs;    /* max distinct input nodes of a merged group (1..24, default 8) */
    uint32_t max_width;     /* max nodes per group (1..32, default 32) */
    uint32_t semantics;     /* PBN_SEM_EQ1 (default) or PBN_SEM_NODEWISE */
    double theta;           /* memory limit of Sec. 3.3 on sum over groups of the
                               number of combined functions (default 65536) */
    uint64_t smem_budget;   /* bytes of plan image that may be staged into shared
                               memory (0 = default 192 KiB); larger tables are read
                               from global memory */
    uint32_t sampler;       /* PBN_PERT_BITSLICED (default) or PBN_PERT_GEOMETRIC */
    uint32_t reserved;
} pbn_group_params;

/* Fill *prm with the defaults above. */
void pbn_group_params_default(pbn_group_params* prm);

/* Build a simulation plan (Algorithm 5, Preparation) for the retained nodes of net.
 * GROUPED: nodes with >= 2 functions are split into m groups, m starting from the
 * lower bound of Eq. 2 and grown by one until the greedy partition of Algorithm 3
 * satisfies sum_i prod_{v in S_i} l(v) <= theta and every group has at most
 * max_inputs distinct inputs and max_width nodes (when only the input or width cap
 * fails, m grows by the number of nodes the greedy could not place); nodes with one
 * function are grouped greedily by most shared parents under the same caps
 * (Algorithm 4).  Each group's functions are merged into one table T[c][x]
 * (Sec. 3.3): c = mixed-radix combined choice, x = packed input pattern, output bit
 * i = node i of the group (right to left).  Groups are packed into 32-bit words of
 * the state (a group never straddles a word); the state is exposed as uint64 words.
 * prm may be NULL (defaults).  On success *out owns a new plan.
 * Errors: PBN_EINVAL, PBN_ETOOBIG (a table exceeds 2^30 bits), PBN_ENOMEM. */
int pbn_group(const pbn_net* net, const pbn_group_params* prm, pbn_plan** out);

typedef struct {
    uint32_t n;              /* original nodes */
    uint32_t n_retained;     /* simulated nodes */
    uint32_t n_groups;       /* groups, i.e. table lookups per non-perturbed step */
    uint32_t n_groups_multi; /* groups made of nodes with >= 2 functions */
    uint32_t state_words;    /* uint64 words per trajectory of the grouped state */
    uint32_t n_sel_blocks;   /* SEL Philox blocks drawn per non-perturbed step */
    uint32_t m_lower_bound;  /* m^_min of Eq. 2 (0 if there are no multi-function nodes) */
    uint32_t m_found;        /* m used by Algorithm 4 for the multi-function nodes */
    uint64_t sum_weights;    /* sum over multi groups of prod l(v) (Sec. 3.3) */
    uint64_t table_bytes;    /* bytes of merged tables */
    uint64_t image_bytes;    /* bytes of the device image (pbn_plan_image) */
    uint64_t stage_bytes;    /* leading bytes of the image staged into shared memory */
    uint32_t tables_in_smem; /* 1 if the tables are staged into shared memory */
    uint32_t total_inputs;   /* input bits gathered per non-perturbed step: each merged group's
                                distinct inputs, plus for a split node the mean in-degree of
                                its functions (one function is evaluated) */
    uint32_t n_multi;        /* retained nodes with >= 2 functions */
    uint32_t total_thresholds; /* selection thresholds below 2^32 over those nodes */
    uint32_t n_split;        /* groups that are one multi-function node whose inputs exceed
                                max_inputs: each of its functions keeps its own table over
                                its own inputs, and the node's choice selects the output */
    uint32_t semantics;      /* PBN_SEM_EQ1 or PBN_SEM_NODEWISE */
    uint32_t sampler;        /* PBN_PERT_BITSLICED or PBN_PERT_GEOMETRIC */
    uint32_t reserved;
    double ops_per_step;     /* algorithmic 32-bit integer operations of one trajectory-step:
                                Philox blocks at 56 ops (9 rounds of 2 mul.hi, 2 mul.lo,
                                2 xor3), 12 per bit-sliced level pair, the expected number of
                                level pairs until every lane of each 64-node word is decided;
                                weighted by the probability (1-p')^n of an unperturbed step:
                                56 per SEL block, 2 per threshold, 1 per multi-function node,
                                3 per group input, 5 per group, 2 per state word; 8 for counts */
} pbn_plan_info;

/* Errors: PBN_EINVAL. */
int pbn_plan_info_get(const pbn_plan* plan, pbn_plan_info* out);

/* Serialise the plan's device image (group specs, thresholds, maps, tables) into
 * host memory host_dst of cap bytes (cap >= image_bytes).  The caller copies it
 * to a device buffer of its own that is 16-byte aligned and passes that buffer to
 * pbn_simulate.  Errors: PBN_EINVAL (NULL or cap too small). */
int pbn_plan_image(const pbn_plan* plan, void* host_dst, size_t cap);

/* Layout of the grouped state: pos[i] (capacity n) = 32 * word32 + bit of
 * original node i in the state, where word32 = 2 * (uint64 word) + (bit >= 32),
 * or UINT32_MAX for a node removed by reduction.  Errors: PBN_EINVAL. */
int pbn_plan_layout(const pbn_plan* plan, uint32_t* pos);

/* Group of every original node (UINT32_MAX if removed), in evaluation order.
 * Errors: PBN_EINVAL. */
int pbn_plan_groups(const pbn_plan* plan, uint32_t* group_of);

/* ---- simulation ----------------------------------------------------------------- */
#define PBN_INIT_KEYED 0u /* s(0) from the INIT draws (step_begin must be 0) */
#define PBN_INIT_STATE 1u /* start from d_state */

typedef struct {
    uint64_t seed;         /* Philox key */
    uint64_t traj_begin;   /* global id of the first trajectory (< 2^48) */
    uint64_t n_traj;       /* trajectories in this call (< 2^31) */
    uint64_t step_begin;   /* index t of the first step: maps s(t) -> s(t+1) */
    uint64_t n_steps;      /* steps in this call (< 2^32; step_begin + n_steps <= 2^48) */
    uint64_t count_from;   /* states s(u) with u >= count_from are counted: those the
                              call produces (u > step_begin), and the keyed s(0) when
                              count_from = 0; a PBN_INIT_STATE call never counts its
                              initial state (the call before it produced and counted
                              it), so calls resumed from d_state add up to one call */
    uint32_t init;         /* PBN_INIT_KEYED or PBN_INIT_STATE */
    uint32_t n_meta;       /* meta-state nodes (1..1024) */
    const uint32_t* meta_ids;  /* host: original ids of the meta-state nodes (retained) */
    const uint8_t* meta_vals;  /* host: required value of each (NULL: all 1) */
    void* d_state;   /* device uint64 [state_words][n_traj], SoA; read if init is
                        PBN_INIT_STATE, always written with s(step_begin + n_steps) */
    void* d_counts;  /* device uint64 [5][n_traj] or NULL: rows V, n00, n01, n10, n11
                        accumulated (+=) over counted states and consecutive counted
                        pairs (z_prev, z) of the meta-state indicator z */
    void* d_pooled;  /* device uint64 [5] or NULL: the same counts summed over the
                        trajectories of this call, accumulated with atomics */
    void* d_status;  /* device uint32 or NULL: ORed with PBN_DEV_* bits on error */
    void* d_trace;   /* device uint64 [n_steps / trace_stride][state_words][n_traj] or NULL:
                        snapshots of the state after every trace_stride-th step of the
                        call (snapshot i after step i * trace_stride + trace_stride - 1
                        of the call; for checking and sampling; slows the kernel) */
    uint32_t lanes_per_traj;   /* lanes cooperating on one trajectory: 0 = auto, 1, 2, 4, 8, 16, 32 */
    uint32_t trajs_per_block;  /* 0 = auto; else a multiple of 32 / lanes_per_traj with
                                  trajs_per_block * lanes_per_traj <= 1024 */
    uint32_t kernel;           /* PBN_KERNEL_AUTO, PBN_KERNEL_INTERP, PBN_KERNEL_COMPILED or PBN_KERNEL_TEAM */
    uint32_t trace_stride;     /* steps between snapshots (0 or 1: every step) */
    uint32_t team_warps;       /* PBN_KERNEL_TEAM: warps per team (0 = auto); trajs_per_block is
                                  then the team's trajectories x the teams per CTA (0 = auto) */
    uint32_t team_trajs_per_lane; /* PBN_KERNEL_TEAM: trajectories per lane, a team of 32 x this
                                  many (0 = auto: 2 when such a team fits, else 1; or 1, 2) */
} pbn_sim_args;

#define PBN_KERNEL_AUTO 0u     /* the compiled plan kernel if pbn_plan_compile succeeded, else the interpreter */
#define PBN_KERNEL_INTERP 1u   /* the generic kernel that reads the plan image */
#define PBN_KERNEL_COMPILED 2u /* the plan's own kernel (compiled on first use) */
/* the team interpreter for wide states: K warps share 32 x TPL trajectories (TPL per
 * lane), splitting each step's perturbation words, SEL blocks and groups, the states
 * in shared memory as [row][trajectory]; Eq. 1 semantics only (node-wise plans:
 * PBN_EINVAL); K x teams per CTA <= 32 */
#define PBN_KERNEL_TEAM 3u

/* Simulate trajectories traj_begin .. traj_begin + n_traj - 1 for steps
 * step_begin .. step_begin + n_steps - 1 (Algorithm 5, ParallelSimulation, with
 * Eq. 1 semantics), enqueued on the CUDA stream `stream` (cudaStream_t, NULL =
 * legacy default stream).  d_image is the caller's 16-byte aligned device copy of
 * pbn_plan_image(plan).  Results are bit-identical to the unreduced, ungrouped
 * definition for any launch shape.  Returns after enqueueing; device-side errors
 * appear in *d_status.  n_traj == 0 enqueues nothing.
 * Errors: PBN_EINVAL (bad pointer, alignment, range, meta node removed or too many
 * distinct meta words (> 16)), PBN_ETOOBIG (shared memory), PBN_ECUDA. */
int pbn_simulate(const pbn_plan* plan, const void* d_image, const pbn_sim_args* args,
                 void* stream);

/* Compile the plan into a kernel of its own (Algorithm 5's Preparation output as
 * constants: group input positions, selection thresholds, the levels of P and the
 * small merged tables become immediates, the state lives in registers), with NVRTC
 * for sm_103a, and keep it with the plan.  Idempotent and thread-safe.  Plans with
 * more than 1024 original nodes, 64 state words or 24 SEL blocks are not compiled
 * (the interpreter kernel runs them).  *compile_ms (may be NULL) receives the host
 * time spent.  Errors: PBN_EINVAL (plan not compilable), PBN_ECUDA (NVRTC missing,
 * compilation or module load failed; pbn_last_error_detail() has the log). */
int pbn_plan_compile(const pbn_plan* plan, uint32_t flags, double* compile_ms);

/* pbn_plan_compile flags.  Default (0): the perturbation words are drawn in pairs
 * by one rolled loop (two independent Philox chains, small code).
 * PBN_COMPILE_PERT_UNROLLED: one word at a time, every level pair unrolled with
 * the bits of P as constants.
 * PBN_COMPILE_INTERLEAVED: the SEL blocks are drawn before the perturbation check
 * and the first three level pairs of every word are straight-line code, so that
 * these Philox chains can be interleaved (more independent work per thread; the
 * SEL draws of perturbed steps are discarded).
 * Every variant consumes the same keyed draws: results are identical.  Compiling
 * with other flags replaces the kernel. */
#define PBN_COMPILE_PERT_UNROLLED 0x1u
#define PBN_COMPILE_INTERLEAVED 0x2u
/* PBN_COMPILE_PIPELINED: software-pipelined steps; the SEL blocks and the first
 * three perturbation level pairs of step t + 1 are drawn while step t's groups are
 * evaluated (every draw is independent of the state), and the evaluation runs in
 * every step with a select keeping s XOR flips in perturbed steps.  Takes
 * precedence over the two flags above. */
#define PBN_COMPILE_PIPELINED 0x4u
/* PBN_COMPILE_MAGIC_GATHER (combines with the others): within a merged group, the
 * 3 to 8 inputs that sit in one state word are gathered by one multiplication
 * ((s & mask) * mul >> shift, with a multiplier found on the host that makes the
 * field an injective index) instead of one shift and mask per bit; the group's table
 * is rebuilt in that index order and the kernel reads its tables from its own
 * array.  Same results. */
#define PBN_COMPILE_MAGIC_GATHER 0x8u
/* PBN_COMPILE_WIDE: plans of up to 2048 nodes and any number of SEL blocks; the
 * groups are evaluated in the order of the SEL blocks they read and each block is
 * drawn just before its first use (the interleaved and pipelined forms do not
 * apply).  Meant for wide networks with few trajectories. */
#define PBN_COMPILE_WIDE 0x10u
/* PBN_COMPILE_WARP_SPLIT: for wide plans (up to 4096 original nodes, 128 state rows,
 * Eq. 1 semantics): a CTA of K warps runs 32 trajectories, one per lane, their states
 * double-buffered in shared memory as [row][lane]; each warp runs straight-line code
 * for its own share of the perturbation word pairs and of the state rows (their SEL
 * blocks and merged groups), with two CTA barriers per step.  K is
 * PBN_COMPILE_WARPS(K) (1..31), or 2 when 0.  Results equal every other form's. */
#define PBN_COMPILE_WARP_SPLIT 0x20u
#define PBN_COMPILE_WARPS(k) (((uint32_t)(k) & 31u) << 8)
/* with PBN_COMPILE_WARP_SPLIT: registers limited so that m (1..7) CTAs fit an SM */
#define PBN_COMPILE_MINCTAS(m) (((uint32_t)(m) & 7u) << 13)
/* with PBN_COMPILE_WARP_SPLIT: groups evaluated in batches of 4^b (b = 0..3) whose
 * state rows are loaded together; ptxas at -O1 instead of its default -O3 */
#define PBN_COMPILE_WS_BATCH(b) (((uint32_t)(b) & 3u) << 16)
#define PBN_COMPILE_WS_O1 0x40000u
/* with PBN_COMPILE_WARP_SPLIT: the SEL blocks drawn before the barrier by one short
 * loop split over the warps, the choices kept as bytes in shared memory (smaller code,
 * no block drawn twice) */
#define PBN_COMPILE_WS_SELSMEM 0x80000u

/* Attributes of the plan's compiled kernel (after pbn_plan_compile): registers per
 * thread, local-memory (spill) bytes per thread and the flags it was compiled with;
 * any pointer may be NULL.  Errors: PBN_EINVAL (NULL plan, plan not compiled),
 * PBN_ECUDA. */
int pbn_plan_compiled_attrs(const pbn_plan* plan, uint32_t* regs, uint32_t* local_bytes, uint32_t* flags);

/* The CUDA source generated for the plan's own kernel: *len receives its length;
 * dst (capacity cap, may be NULL) receives it NUL-terminated.
 * Errors: PBN_EINVAL (plan not compilable, cap too small). */
int pbn_plan_source(const pbn_plan* plan, uint32_t flags, char* dst, size_t cap, size_t* len);

/* ---- batched form: many networks, one persistent launch ------------------------------ */
typedef struct pbn_batch pbn_batch;

typedef struct {
    const pbn_plan* plan;      /* plan of this network (kept alive by the caller) */
    const void* d_image;       /* caller's 16-byte aligned device copy of pbn_plan_image(plan) */
    uint64_t seed;             /* Philox key of this network's draws */
    uint64_t traj_begin;       /* global id of its first trajectory (< 2^48) */
    uint64_t n_traj;           /* trajectories (1 .. 2^31 - 1) */
    uint64_t step_begin;       /* index of its first step */
    uint64_t count_from;       /* states s(u) with u >= count_from are counted (as in
                                  pbn_sim_args: launches resumed from d_state add up) */
    uint32_t init;             /* PBN_INIT_KEYED (step_begin must be 0) or PBN_INIT_STATE */
    uint32_t n_meta;           /* meta-state nodes (1..1024, retained, within 16 state words) */
    const uint32_t* meta_ids;  /* host */
    const uint8_t* meta_vals;  /* host, NULL = all 1 */
    void* d_state;             /* device uint64 [state_words][n_traj] */
    void* d_counts;            /* device uint64 [5][n_traj] or NULL (accumulated) */
    void* d_pooled;            /* device uint64 [5] or NULL (accumulated) */
} pbn_batch_net;

typedef struct {
    uint32_t n_nets;
    uint32_t n_items;          /* work items: trajectory ranges of one network, each as
                                  many trajectory slots as fit in shared memory, at
                                  most `threads` / (the network's lanes per trajectory),
                                  or 2 x `threads` for teams of two trajectories per lane */
    uint32_t threads;          /* threads per CTA */
    uint32_t max_lanes;        /* the most lanes per trajectory any network of the batch uses
                                  (32 for a team: every lane of its warps works on it) */
    uint64_t desc_bytes;       /* bytes of pbn_batch_image */
    uint64_t smem_bytes;       /* dynamic shared memory per CTA */
    double est_ops_per_step;   /* sum over networks of n_traj x ops_per_step */
    uint32_t n_compiled;       /* networks run by compiled code (pbn_batch_compile) */
    uint32_t n_items_compiled; /* split batches: the compiled networks' work items */
    uint32_t n_team;           /* interpreted networks run by the team interpreter */
    uint32_t reserved;         /* 0 */
} pbn_batch_info;

/* Describe a batch of networks for the persistent work-queue kernel: each network
 * gets its staging mode (specs and tables, specs only, or none in shared memory), its
 * trajectory slots per work item and its interpreter (teams of warps on 32 or 64
 * trajectories for states of 8 rows or more, else 1-32 lanes per trajectory; see
 * pbn_batch_create_ex), is cut into work items of that many trajectories, and the
 * items are ordered by descending estimated work.  The networks' plans and device buffers must stay
 * valid while the batch is used.  On success *out owns the batch (pbn_batch_free).
 * Errors: PBN_EINVAL (missing or misaligned buffer, range, meta node), PBN_ETOOBIG
 * (a network's specs and trajectory rows exceed the per-CTA shared memory),
 * PBN_ENOMEM. */
int pbn_batch_create(const pbn_batch_net* nets, uint32_t n_nets, pbn_batch** out);
/* pbn_batch_create with a choice of CTA size for the interpreted batch kernel: 512
 * (as pbn_batch_create) or 1024 threads (64 registers a thread: twice the warps per
 * SM, for wide networks' lane groups; such a batch cannot be compiled).
 * Errors: as pbn_batch_create, PBN_EINVAL for another CTA size. */
int pbn_batch_create_cta(const pbn_batch_net* nets, uint32_t n_nets, uint32_t threads, pbn_batch** out);
/* pbn_batch_create_cta with flags.  By default an interpreted network whose state
 * has 8 rows or more (Eq. 1 semantics) runs the team interpreter (PBN_KERNEL_TEAM's
 * loop: teams of warps on 32 trajectories, as many teams per work item as shared
 * memory holds, the CTA's warps split evenly over them); PBN_BATCH_LANE_GROUPS keeps
 * every interpreted network on lane groups.  The choice holds for the split batches
 * pbn_batch_compile makes.  Errors: as pbn_batch_create_cta, PBN_EINVAL for unknown
 * flags. */
#define PBN_BATCH_LANE_GROUPS 0x1u
int pbn_batch_create_ex(const pbn_batch_net* nets, uint32_t n_nets, uint32_t threads, uint32_t flags,
                        pbn_batch** out);
int pbn_batch_info_get(const pbn_batch* batch, pbn_batch_info* out);

/* Give the batch compiled code (the batched form of Algorithm 5 with each network's
 * Preparation output as constants, as pbn_plan_compile does for one network): every
 * network whose plan compiles with `flags` (PBN_COMPILE_PERT_UNROLLED,
 * PBN_COMPILE_INTERLEAVED, PBN_COMPILE_PIPELINED, PBN_COMPILE_WIDE; multiply gathers
 * are not offered here) becomes a device function of one generated module, with its
 * Philox keys and meta-state rows as constants, run one trajectory per thread (at
 * most 96 networks per module, those with the most work: the CUDA 13.0 linker
 * crashed on a module of 136 network functions); a
 * persistent kernel in the same module pops the work items from the device queue and
 * calls the network's function, or, for networks that do not compile, the
 * interpreter (prebuilt relocatable device code, pbn_batch_item.cubin next to the
 * library, linked with nvJitLink).  Call it before pbn_batch_image: it re-cuts the
 * compiled networks' work items (pbn_batch_info_get gives the new n_items,
 * desc_bytes, smem_bytes and n_compiled).  Results are bit-identical to the
 * uncompiled batch.  *compile_ms (may be NULL) receives the host time.  Host memory
 * and one CUDA library owned by the batch; no device memory is allocated.
 * Errors: PBN_EINVAL (NULL, compiled already, a batch of 1,024-thread CTAs,
 * unsupported flags, no network compiles), PBN_ECUDA (NVRTC, nvJitLink or loading
 * failed), PBN_ENOMEM. */
int pbn_batch_compile(pbn_batch* batch, uint32_t flags, double* compile_ms);
/* Option of pbn_batch_compile (ORed into flags): a split batch.  The module holds
 * only the compiled networks' functions; the other networks' items are shaped for
 * the library's interpreter kernel of 1,024-thread CTAs.  Each run is then two
 * persistent launches on the same queue and stream (the compiled networks' items,
 * then the others), so that compiled code keeps its registers and the interpreter
 * its warps. */
#define PBN_BATCH_SPLIT 0x80000000u

/* Serialise the batch's device table (network descriptors, then work items) into
 * host memory (cap >= desc_bytes); the caller copies it to a 16-byte aligned device
 * buffer.  Errors: PBN_EINVAL. */
int pbn_batch_image(const pbn_batch* batch, void* host_dst, size_t cap);

/* One persistent launch on `stream`: every network advances n_steps steps, from
 * step_begin + step_offset (keyed initial states only when step_offset == 0), with
 * the same results as pbn_simulate on each network alone.  d_queue is caller scratch
 * of two uint32 counters (the next work item and the CTAs that found the queue
 * empty) that must be zero before the first launch; the last CTA of every launch
 * resets them, so launches can follow each other (or be captured in a CUDA graph)
 * without a reset.  Launches sharing one d_queue must not overlap.  ctas_per_sm = 0
 * uses the occupancy limit.  d_status (may be NULL) receives PBN_DEV_* bits.  The
 * kernel's shared-memory limit is raised on the current device as the batch needs
 * and never lowered, and the occupancy is found once per batch and device, so
 * batches, devices and this call and pbn_batch_run_static may be mixed freely.
 * Errors: PBN_EINVAL, PBN_ETOOBIG, PBN_ECUDA. */
int pbn_batch_run(const pbn_batch* batch, const void* d_desc, uint32_t* d_queue, uint64_t step_offset,
                  uint64_t n_steps, uint32_t ctas_per_sm, uint32_t* d_status, void* stream);
void pbn_batch_free(pbn_batch* batch);

/* Same launch as pbn_batch_run, for callers that cannot allocate device memory when
 * they run a batch (an allocator that owns the device, a CUDA graph being recorded,
 * a latency-critical loop that must not call cudaMalloc or cudaFree, which can
 * synchronise the device).  The paper has no counterpart: this is a deployment
 * option of the batched form.  The work-queue scratch comes from a static array the
 * library keeps in device memory: PBN_STATIC_QUEUE_SLOTS queues of two uint32
 * counters, selected by `slot`; the call clears its slot (cudaMemsetAsync on
 * `stream`) before the launch and allocates nothing.  Calls that use the same slot
 * and overlap on the GPU race; concurrent batches must use different slots.  The
 * first call on a device looks up the array's device address (once per device, with
 * that device current), so make that first call before any stream capture.
 * Errors: PBN_EINVAL (slot >= PBN_STATIC_QUEUE_SLOTS, NULL or misaligned table,
 * range), PBN_ETOOBIG, PBN_ECUDA. */
#define PBN_STATIC_QUEUE_SLOTS 16u
int pbn_batch_run_static(const pbn_batch* batch, const void* d_desc, uint32_t slot, uint64_t step_offset,
                         uint64_t n_steps, uint32_t ctas_per_sm, uint32_t* d_status, void* stream);

/* ---- estimation ------------------------------------------------------------------ */
typedef struct {
    double alpha;        /* n01 / (n00 + n01), NaN if undefined */
    double beta;         /* n10 / (n10 + n11), NaN if undefined */
    double pi;           /* V / L, the steady-state probability estimate */
    double var;          /* alpha beta (2 - alpha - beta) / ((alpha + beta)^3 L) */
    double z;            /* Phi^-1((1 + s) / 2) */
    double n_star_real;  /* alpha beta (2-alpha-beta)/(alpha+beta)^3 (z/r)^2 */
    uint64_t L;          /* counted states: n00 + n01 + n10 + n11 + n_traj */
    uint64_t m_star;     /* burn-in; UINT64_MAX if undefined */
    uint64_t n_star;     /* required counted states; UINT64_MAX if undefined */
    int32_t defined;     /* 1 if alpha, beta > 0 and both are defined */
    int32_t done;        /* 1 if defined, L >= n_star and burn_in_used >= m_star */
} pbn_estimate_out;

/* Two-state Markov chain estimate (Sec. 4.2, the Raftery-Lewis approach the paper
 * cites): from the pooled counts [V, n00, n01, n10, n11] of n_traj trajectories,
 * precision r, confidence s and burn-in tolerance eps:
 *   m* = max(1, ceil(log(eps (alpha+beta) / max(alpha, beta)) / log|1-alpha-beta|))
 *        (1 if alpha + beta = 1; undefined if |1 - alpha - beta| = 1),
 *   N* = ceil(alpha beta (2 - alpha - beta) / (alpha + beta)^3 (z / r)^2).
 * burn_in_used is the number of initial states the caller excluded per trajectory.
 * Errors: PBN_EINVAL (NULL, r <= 0, s not in (0,1), eps <= 0, n_traj == 0). */
int pbn_estimate(const uint64_t counts[5], uint64_t n_traj, uint64_t burn_in_used,
                 double r, double s, double eps, pbn_estimate_out* out);

/* ---- misc ------------------------------------------------------------------------ */
const char* pbn_strerror(int status);
const char* pbn_last_error_detail(void);
void pbn_net_free(pbn_net* net);
void pbn_plan_free(pbn_plan* plan);
/* Library version string. */
const char* pbn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PBN_H */
