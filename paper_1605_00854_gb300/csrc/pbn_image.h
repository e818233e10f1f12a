/*
 * pbn_image.h -- device image of a simulation plan (internal to the library).
 *
 * The image is one contiguous, 16-byte aligned byte buffer the caller uploads to
 * device memory.  Its leading `stage_bytes` are bulk-copied into each CTA's shared
 * memory at kernel start; when the merged tables do not fit, they stay in global
 * memory (L2-resident) and only the specs are staged.
 *
 * Sections (byte offsets in pbn_img_header, each 16-byte aligned):
 *   words   [W32]        uint2 {first group, number of groups} of state word k
 *   groups  [n_groups]   pbn_img_group, sorted by output word
 *   multi   [n_multi]    pbn_img_multi, the multi-function nodes of each group in
 *                        group bit order
 *   thr     [...]        uint32 selection thresholds T_j < 2^32 (Sec. 2.2 via
 *                        integer cumulative thresholds)
 *   inputs  [...]        uint32 input records, 4 per chunk, each group starting a
 *                        chunk and padded with records of the always-zero row
 *                        W32: (4 * row) << 5 | rot, where row is the state word
 *                        holding input b and rot = (bit - b mod 4) mod 32 rotates
 *                        that bit to position b mod 4 of its chunk
 *   selblk  [n_sel]      uint32 SEL block indices r / 4 drawn per step
 *   ret     [W]          uint64 mask of retained lanes of original word w
 *   pos     [n]          uint32 state position (32 * row + bit) of original node i,
 *                        0xFFFFFFFF for a leaf
 *   tables  [...]        uint32 words of packed table entries; entry e of a group
 *                        with log2 entry width l2w occupies bits
 *                        [e << l2w, (e + 1) << l2w) of its table
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
    uint32_t off_words, off_groups, off_multi, off_thr;
    uint32_t off_inputs, off_selblk, off_ret, off_pos;
    uint32_t off_tables;
    uint32_t image_bytes;
    uint32_t stage_bytes;
    uint32_t tables_in_smem;
} pbn_img_header; /* 80 bytes */

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
    uint32_t u_off;     /* bits 0..23: byte offset of the node's SEL uniform in a
                           trajectory's uniform row (4 * (4 * selblk index + rank mod 4));
                           bits 24..31: number of thresholds below 2^32 */
    uint32_t radix;     /* mixed-radix weight of this node's choice */
    uint32_t t1, t2;    /* the thresholds when there are at most two; otherwise t1 is
                           the index of the first one in the thresholds section */
} pbn_img_multi; /* 16 bytes */

#endif
