"""The large-database recipe: genera of bacterial-like genomes plus
repeat-rich eukaryote-like genomes whose repeated segments overfill buckets
(bucket cap, overflow counts).  A reduced instance is checked against the
oracle in full; the scaled instance (about 15 Gbp) is built at full size and
checked on a key range against buckets recomputed on the host from the
sketches of all windows."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import dev, gpu_build, gpu_classify, host_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2106_08150_gb300 import mc as m
    m.use_torch_allocator()
    return m


def test_repeat_rich_database_and_classification_match_oracle(mc):
    w = synth.large_workload(seed=91, n_pairs=3000, n_families=1, genera_per_family=2, n_euk=4, len_scale=0.02,
                             euk_scale=0.03)
    p = dict(w.db_params, bucket_cap=4)
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, splits=[7, 20], **p)
    odb = oracle.DB(w.genomes, w.goffs, **p)
    try:
        gk, gc, gl = db.dump()
        ok, oc, ol = odb.dump()
        assert len(gk) == len(ok) and (gk == ok).all() and (gc == oc).all() and (gl == ol).all()
        st, ost = db.stats(), odb.stats()
        for k in ["n_windows", "n_pairs", "n_keys", "n_locations", "overflow_keys"]:
            assert st[k] == ost[k], k
        assert st["overflow_keys"] > 100  # the repeats overfill buckets
        got = gpu_classify(mc, db, w.reads, w.roffs, w.qoffs, **{k: v for k, v in w.cls_params.items()
                                                                  if k != "max_candidates"})
        want = odb.classify(w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, n_threads=8, **w.cls_params)
        for a, b in zip(got[:3], want):
            assert (a == b).all()
    finally:
        db.free()


def test_scaled_large_database_key_range(mc):
    """Full-size build of the scaled recipe; the buckets of one key range
    must equal those recomputed on the host from every window's sketch
    (sorted locations, the cap smallest kept)."""
    import torch
    w = synth.large_workload(seed=1002, scaled=True, n_pairs=1000)
    p = w.db_params
    d_g, d_o = dev(w.genomes), dev(w.goffs)
    db = mc.Database.create(w.parent, **p)
    try:
        db.add_targets(d_g, d_o, w.taxon_of_target)
        db.finalize()
        st = db.stats()
        lens = np.diff(w.goffs).astype(np.int64)
        k, stride = p["k"], p["window_stride"]
        nw = np.where(lens >= k, (lens - k + stride) // stride, 0)
        assert st["n_windows"] == int(nw.sum())
        assert st["overflow_keys"] > 0 and st["n_locations"] + st["dropped_locations"] == st["n_pairs"]
        assert 0 < st["load_factor"] <= 0.5
        # sketches of all windows, selected on the device for one key range
        lo, hi = 0, (1 << 32) // 4096
        n_seq = len(w.goffs) - 1
        prm = mc.db_params(**p)
        win = torch.zeros(n_seq + 1, dtype=torch.int64, device="cuda")
        mc.mc_window_offsets(prm, n_seq, d_o, win)
        n_win = int(win[-1].item())
        s = p["sketch_size"]
        sk = torch.zeros(n_win * s, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(n_win, dtype=torch.int32, device="cuda")
        mc.mc_sketch(prm, n_seq, d_g, d_o, win, n_win, sk, cnt)
        torch.cuda.synchronize()
        pos = torch.arange(s, device="cuda").repeat(n_win)
        valid = pos < cnt.repeat_interleave(s)
        u = sk.to(torch.int64) & 0xFFFFFFFF
        sel = valid & (u >= lo) & (u < hi)
        idx = torch.nonzero(sel).squeeze(1)
        feats = u[idx].cpu().numpy().astype(np.uint32)
        gwin = (idx // s).cpu().numpy().astype(np.int64)
        del sk, cnt, u, sel, idx, pos, valid
        wb = win.cpu().numpy().astype(np.int64)
        tgt = np.searchsorted(wb, gwin, side="right") - 1
        loc = (tgt.astype(np.uint64) << np.uint64(32)) | (gwin - wb[tgt]).astype(np.uint64)
        order = np.lexsort((loc, feats))
        feats, loc = feats[order], loc[order]
        keys, first, counts = np.unique(feats, return_index=True, return_counts=True)
        cap = p["bucket_cap"]
        keep = np.concatenate([np.arange(f, f + min(c, cap)) for f, c in zip(first, counts)])
        gk, gc, gl = db.dump(lo, hi)
        assert len(gk) == len(keys) > 1000
        assert (gk == keys).all()
        assert (gc == np.minimum(counts, cap)).all()
        assert (gl == loc[keep]).all()
        assert (counts > cap).any()
    finally:
        db.free()
