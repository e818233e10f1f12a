"""Test helper: decode a plan's device image (layout of csrc/pbn_image.h) in Python."""
import struct

import numpy as np

HEADER_FIELDS = ["magic", "n", "W", "W32", "n_groups", "n_multi", "n_sel", "P",
                 "off_words", "off_groups", "off_multi", "off_selslot", "off_thr", "off_inputs",
                 "off_selblk", "off_gorder", "off_wgroups", "off_subs", "off_tables", "off_ret", "off_pos", "image_bytes",
                 "stage_bytes", "tables_in_smem", "semantics", "sampler", "off_geo"]


def decode(img: np.ndarray) -> dict:
    b = img.tobytes()
    H = dict(zip(HEADER_FIELDS, struct.unpack_from("<27I", b, 0)))
    u32 = np.frombuffer(b, dtype=np.uint32)
    words = u32[H["off_words"] // 4: H["off_words"] // 4 + 2 * H["W32"]].reshape(-1, 2)
    groups = []
    for g in range(H["n_groups"]):
        tab_off, in_chunk, mul_first, q, l2w, n_mul, shift = struct.unpack_from(
            "<3I4B", b, H["off_groups"] + 16 * g)
        groups.append(dict(tab_off=tab_off, in_chunk=in_chunk, mul_first=mul_first, q=q, l2w=l2w,
                           n_mul=n_mul, shift=shift))
    multi = []
    for m in range(H["n_multi"]):
        ch_off, radix = struct.unpack_from("<2I", b, H["off_multi"] + 8 * m)
        rec = (ch_off % 4) * H["n_sel"] + ch_off // 4   # slot record layout: (slot mod 4) * n_sel + slot / 4
        t1, t2, n_thr, first = struct.unpack_from("<4I", b, H["off_selslot"] + 16 * rec)
        multi.append(dict(u_slot=ch_off, n_thr=n_thr, radix=radix, t1=t1, t2=t2, first=first))
    sel = u32[H["off_selblk"] // 4: H["off_selblk"] // 4 + H["n_sel"]]
    pos = u32[H["off_pos"] // 4: H["off_pos"] // 4 + H["n"]]
    ret = np.frombuffer(b, dtype=np.uint64)[H["off_ret"] // 8: H["off_ret"] // 8 + H["W"]]
    return dict(H=H, u32=u32, words=words, groups=groups, multi=multi, sel=sel, pos=pos, ret=ret)


def thresholds(D, m):
    M = D["multi"][m]
    if M["n_thr"] <= 2:
        return [M["t1"], M["t2"]][: M["n_thr"]]
    o = D["H"]["off_thr"] // 4 + M["first"]
    return [int(v) for v in D["u32"][o: o + M["n_thr"]]]


STRIDE = 32  # row-interleaved records: chunk j, multi m, function f of a group are 32 apart


def multi_index(G, m):
    """Index of the m-th multi-function record of group record G."""
    return G["mul_first"] + STRIDE * m


def inputs(D, g):
    """(row, bit) of each input b of group g, decoded from its chunked records."""
    G = D["groups"][g]
    out = []
    for b in range(G["q"]):
        o = D["H"]["off_inputs"] // 4 + 4 * (G["in_chunk"] + STRIDE * (b // 4)) + (b & 3)
        rec = int(D["u32"][o])
        row, rot = rec >> 7, rec & 31
        out.append((row, ((b & 3) + rot) & 31))
    return out


def word_groups(D, w):
    """Group indices of state word w."""
    first, cnt = (int(x) for x in D["words"][w])
    o = D["H"]["off_wgroups"] // 4 + first
    return [int(x) for x in D["u32"][o: o + cnt]]


SPLIT = 0xFF


def subs(D, g):
    """Sub-function records (in_chunk, k, tab_off) of split group g, one per function."""
    G = D["groups"][g]
    out = []
    for j in range(G["q"]):
        o = D["H"]["off_subs"] // 4 + 2 * (G["tab_off"] + STRIDE * j)
        a, tab_off = int(D["u32"][o]), int(D["u32"][o + 1])
        out.append((a & 0x7FFFFFF, a >> 27, tab_off))
    return out


def sub_inputs(D, in_chunk, k):
    o = D["H"]["off_inputs"] // 4 + 4 * in_chunk
    out = []
    for b, rec in enumerate(int(v) for v in D["u32"][o: o + k]):
        row, rot = rec >> 7, rec & 31
        out.append((row, ((b & 3) + rot) & 31))
    return out


def sub_entry(D, tab_off, x):
    w = int(D["u32"][D["H"]["off_tables"] // 4 + tab_off + (x >> 5)])
    return (w >> (x & 31)) & 1


def entry(D, g, e):
    G = D["groups"][g]
    bo = e << G["l2w"]
    w = int(D["u32"][D["H"]["off_tables"] // 4 + G["tab_off"] + (bo >> 5)])
    return (w >> (bo & 31)) & ((1 << (1 << G["l2w"])) - 1)
