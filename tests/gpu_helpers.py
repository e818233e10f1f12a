"""Test helpers that run the CUDA path and bring results back in original node order."""
import numpy as np

from paper_1605_00854_gb300 import api


def plan_for(text, interest=(0, 1, 2), mode=0, reduce=True, **kw):
    net = api.Net.load(text)
    if reduce:
        net, ids = net.reduce(list(interest))
    else:
        ids = np.arange(net.info().n, dtype=np.uint32)
    return api.Plan(net, mode=mode, **kw), ids


def run(plan, *, seed, n_traj, n_steps, meta, meta_vals=None, traj_begin=0, step_begin=0,
        count_from=0, init_bits=None, trace=False, lanes=0, tpb=0, chunks=None, kernel=0, team_warps=0,
        team_tpl=0):
    """Run pbn_simulate; returns dict(final bits [T, n], counts [T, 5] uint64,
    pooled [5], status, trace bits [T, S, n] or None).  `chunks` splits the steps into
    consecutive launches resumed from the device state."""
    import torch
    dev = "cuda"
    bufs = api.alloc_buffers(plan, n_traj, dev)
    init = None
    if init_bits is not None:
        bufs.state.copy_(torch.from_numpy(pack(plan, init_bits).view(np.int64)).to(dev))
        init = 1
    tr = None
    if trace:
        tr = torch.zeros((n_steps, plan.info.state_words, n_traj), dtype=torch.int64, device=dev)
    chunks = chunks or [n_steps]
    assert sum(chunks) == n_steps
    sb = step_begin
    for i, c in enumerate(chunks):
        api.simulate(plan, bufs, seed=seed, n_steps=c, meta_ids=meta, meta_vals=meta_vals,
                     traj_begin=traj_begin, step_begin=sb, count_from=count_from,
                     init=(init if i == 0 else 1), lanes_per_traj=lanes, trajs_per_block=tpb,
                     kernel=kernel, team_warps=team_warps, team_trajs_per_lane=team_tpl,
                     trace=None if tr is None else tr[sb - step_begin: sb - step_begin + c])
        sb += c
    torch.cuda.synchronize()
    out = {
        "final": plan.unpack(bufs.state.cpu().numpy().view(np.uint64)),
        "counts": bufs.counts.cpu().numpy().view(np.uint64).T.copy(),
        "pooled": bufs.pooled.cpu().numpy().view(np.uint64).copy(),
        "status": int(bufs.status.cpu().item()),
        "trace": None,
    }
    if tr is not None:
        t = tr.cpu().numpy().view(np.uint64)
        out["trace"] = np.stack([plan.unpack(t[s]) for s in range(n_steps)], axis=1)
    return out


def pack(plan, bits):
    """bits [T, n] in original order -> grouped state words [state_words, T] uint64."""
    pos = plan.layout()
    T = bits.shape[0]
    words = np.zeros((plan.info.state_words, T), dtype=np.uint64)
    for i, p in enumerate(pos):
        if p == 0xFFFFFFFF:
            continue
        row, bit = int(p) >> 5, int(p) & 31
        sh = np.uint64(bit + 32 * (row & 1))
        words[row >> 1] |= bits[:, i].astype(np.uint64) << sh
    return words
