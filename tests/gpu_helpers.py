"""Helpers for the GPU tests: move synthetic workloads to the device and run
the CUDA path through the C ABI."""
import numpy as np


def dev(a, torch_dtype=None):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    t = torch.from_numpy(a).to("cuda")
    return t if torch_dtype is None else t.to(torch_dtype)


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def u8(s):
    if isinstance(s, str):
        return np.frombuffer(s.encode(), dtype=np.uint8).copy()
    return np.ascontiguousarray(s, dtype=np.uint8)


def offsets(lengths):
    o = np.zeros(len(lengths) + 1, dtype=np.uint64)
    o[1:] = np.cumsum(lengths)
    return o


def gpu_sketch(mc, seq, offs, **p):
    """(win_offs, sketch[n_win, s], cnt) from the CUDA sketch kernel."""
    import torch
    prm = mc.db_params(**p)
    n_seq = len(offs) - 1
    d_seq = dev(u8(seq)) if len(seq) else torch.zeros(1, dtype=torch.uint8, device="cuda")
    d_offs = dev(offs)
    d_win = torch.zeros(n_seq + 1, dtype=torch.int64, device="cuda")
    mc.mc_window_offsets(prm, n_seq, d_offs, d_win)
    win = d_win.cpu().numpy().view(np.uint64)
    n_win = int(win[-1])
    s = p["sketch_size"]
    d_sk = torch.zeros(max(1, n_win * s), dtype=torch.int32, device="cuda")
    d_cnt = torch.zeros(max(1, n_win), dtype=torch.int32, device="cuda")
    mc.mc_sketch(prm, n_seq, d_seq, d_offs, d_win, n_win, d_sk, d_cnt)
    torch.cuda.synchronize()
    return win, host_u32(d_sk)[: n_win * s].reshape(n_win, s), host_u32(d_cnt)[:n_win]


def gpu_build(mc, w_genomes, w_goffs, parent, taxon, splits=None, finalize_each=False, **p):
    """Database from targets, optionally added in several calls."""
    db = mc.Database.create(parent, **p)
    n = len(w_goffs) - 1
    bounds = [0, n] if splits is None else [0, *splits, n]
    for a, b in zip(bounds[:-1], bounds[1:]):
        lo, hi = int(w_goffs[a]), int(w_goffs[b])
        seq = dev(w_genomes[lo:hi]) if hi > lo else dev(np.zeros(1, np.uint8))
        offs = dev((w_goffs[a:b + 1] - np.uint64(lo)).astype(np.uint64))
        first = db.add_targets(seq, offs, taxon[a:b])
        assert first == a
        if finalize_each:
            db.finalize()
    db.finalize()
    return db


def gpu_classify(mc, db, reads, roffs, qoffs, with_cands=False, m=4, **cp):
    import torch
    nq = len(qoffs) - 1
    d_r = dev(u8(reads)) if len(reads) else dev(np.zeros(1, np.uint8))
    cands = torch.zeros(max(1, nq * m * 4), dtype=torch.int32, device="cuda") if with_cands else None
    counters = torch.zeros(mc.MC_DEBUG_COUNTERS, dtype=torch.int64, device="cuda")
    label, hits, top = db.classify(d_r, dev(roffs), dev(qoffs), cands=cands, counters=counters,
                                   max_candidates=m, **cp)
    mc.mc_classify_status(db.handle)
    out = [host_u32(label), host_u32(hits), host_u32(top)]
    if with_cands:
        out.append(host_u32(cands)[: nq * m * 4].reshape(nq, m, 4))
    out.append(counters.cpu().numpy())
    return out
