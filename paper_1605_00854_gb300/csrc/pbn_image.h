/*
 * pbn_image.h -- device image of a simulation plan (internal to the library).
 *
 * The image is one contiguous, 16-byte aligned byte buffer the caller uploads to
 * device memory.  Its leading `stage_bytes` are bulk-copied into each CTA's shared
 * memory at kernel start; when the merged tables do not fit, they stay in global
 * memory (L2-resident) and only the specs are staged.
 *
 * Sections (byte offsets in pbn_img_header, each 16-byte aligned):
 *   words   [W32]        uint2 {first, count}: range of wgroups listing the groups of
 *                        state word k
 *   groups  [n_groups]   pbn_img_group in evaluation (shape) order: groups sorted by
 *                        split first, then input chunks and multi-function nodes
 *                        descending, so that groups taken together look alike;
 *                        within a shape class the groups of different output words
 *                        alternate (the i-th group of every word before any
 *                        (i+1)-th), so lanes taking consecutive groups write
 *                        different words
 *   multi   [...]        pbn_img_multi, the multi-function nodes of each group in
 *                        group bit order: where their choice is and its radix
 *
 * Row-interleaved records: the records a group reads are laid out in rows of 32
 * consecutive groups with a stride of 32, so that lanes taking consecutive groups
 * read consecutive records: input chunk j of group k = 32 r + l is chunk
 * in_chunk + 32 j (in_chunk = base_r + l); multi record m is mul_first + 32 m;
 * function f of a split node is record tab_off + 32 f.  A split node's functions
 * keep their own input chunks contiguous (stride 1) after the rows.
 *   selslot [4 n_sel]    uint4 {t1, t2, n_thr, thr_first} per SEL slot (4 per drawn
 *                        block, slot = 4 * block index + rank mod 4), stored at
 *                        (slot mod 4) * n_sel + slot / 4: the node's integer
 *                        thresholds (inline when n_thr <= 2); n_thr = 0 for a slot
 *                        without a retained multi-function node
 *   thr     [...]        uint32 selection thresholds T_j < 2^32 of every slot
 *   inputs  [...]        uint32 input records, 4 per chunk, each group starting a
 *                        chunk and padded with records of the always-zero row
 *                        W32: (4 * row) << 5 | rot, where row is the state word
 *                        holding input b and rot = (bit - b mod 4) mod 32 rotates
 *                        that bit to position b mod 4 of its chunk
 *   selblk  [n_sel]      uint32 SEL block indices r / 4 drawn per step, in an order
 *                        that puts the choice words read by one row of 32 groups in
 *                        different shared-memory banks where possible (slots and
 *                        multi records refer to positions in this list)
 *   gorder  [n_groups]   uint32 group index | output word << 20 of group k (the group
 *                        index is k: records are stored in this order)
 *   wgroups [n_groups]   uint32 group indices of each state word (ranges in words)
 *   subs    [...]        uint2 function records of split nodes (see below)
 *   tables  [...]        uint32 words of packed table entries; entry e of a group
 *                        with log2 entry width l2w occupies bits
 *                        [e << l2w, (e + 1) << l2w) of its table
 *   ret     [W]          uint64 mask of retained lanes of original word w
 *   pos     [n]          uint32 state position (32 * row + bit) of original node i,
 *                        0xFFFFFFFF for a leaf
 *   geo     [64]         uint64 thresholds G[k] of the geometric perturbation sampler
 * ret and pos serve only the initial state and perturbed steps and are read from
 * global memory; the staged prefix ends at off_tables (specs) or off_ret (specs
 * and tables).
 */
#ifndef PBN_IMAGE_H
#define PBN_IMAGE_H

#include <stdint.h>

#define PBN_IMG_MAGIC 0x31424E50u /* "PBN1" */

typedef struct {
    uint32_t magic;
    uint32_t n;          /* original nodes */
    uint32_t W;          /* original 64-lane words = ceil(n / 64) */
    uint32_t W32;        /* 32-bit state words (even) */
    uint32_t n_groups;
    uint32_t n_multi;    /* multi records */
    uint32_t n_sel;      /* SEL blocks per step */
    uint32_t P;          /* perturbation threshold */
    uint32_t off_words, off_groups, off_multi, off_selslot, off_thr;
    uint32_t off_inputs, off_selblk, off_gorder, off_wgroups, off_subs, off_tables, off_ret, off_pos;
    uint32_t image_bytes;
    uint32_t stage_bytes;
    uint32_t tables_in_smem;
    uint32_t semantics;  /* PBN_SEM_EQ1 or PBN_SEM_NODEWISE */
    uint32_t sampler;    /* PBN_PERT_BITSLICED or PBN_PERT_GEOMETRIC */
    uint32_t off_geo;    /* uint64 [64] thresholds of the geometric sampler (global) */
} pbn_img_header; /* 108 bytes */

/* A group record with l2w == PBN_IMG_SPLIT is a split node: one multi-function node
 * whose q functions each keep their own table of 2^k one-bit entries over their own
 * k inputs; tab_off is then the index of its first function record
 * (uint2 {first input chunk | k << 27, table offset in words}) and the node's choice
 * selects which function is evaluated. */
#define PBN_IMG_SPLIT 0xFFu

typedef struct {
    uint32_t tab_off;   /* table offset in uint32 words from the tables section */
    uint32_t in_chunk;  /* first 4-record input chunk */
    uint32_t mul_first; /* first multi record */
    uint8_t q;          /* number of inputs */
    uint8_t l2w;        /* log2 of entry bits (0..5) */
    uint8_t n_mul;      /* multi-function nodes in the group */
    uint8_t shift;      /* bit offset of the group in its output word */
} pbn_img_group; /* 16 bytes */

typedef struct {
    uint32_t ch_off;    /* SEL slot of the node = byte offset of its choice in a
                           trajectory's choice row */
    uint32_t radix;     /* mixed-radix weight of this node's choice */
} pbn_img_multi; /* 8 bytes */

#endif
