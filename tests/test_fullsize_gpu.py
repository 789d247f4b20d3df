"""Full-size parity on the mid workload (1,000 genomes, ~3.4 Gbp; 10M read
pairs), in the launch configuration bench.py times: one database build and
one mc_classify call over all pairs with the autotuner's launch shape.

The oracle cannot build the whole database in test time, so it builds the
buckets of a sample of features only (its key filter): every feature of
2,000 randomly sampled queries plus every feature in one key range.  For
those features the oracle's buckets are complete, so the sampled queries'
labels, hit counts and top targets, and the database dump of the key range,
must match exactly."""
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import dev, host_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mid():
    return synth.mid_workload(seed=1001)


def test_fullsize_sampled_parity(mid):
    import torch
    from paper_2106_08150_gb300 import mc

    w = mid
    mc.use_torch_allocator()
    db = mc.Database.create(w.parent, **w.db_params)
    try:
        db.add_targets(dev(w.genomes), dev(w.goffs), w.taxon_of_target)
        db.finalize()
        st = db.stats()
        nq = w.n_queries
        label = torch.empty(nq, dtype=torch.int32, device="cuda")
        hits = torch.empty(nq, dtype=torch.int32, device="cuda")
        top = torch.empty(nq, dtype=torch.int32, device="cuda")
        cp = mc.classify_params(**w.cls_params)
        d_reads, d_roffs, d_qoffs = dev(w.reads), dev(w.roffs), dev(w.qoffs)
        # the launch configuration the bench times: the autotuner's shape
        n_s = 1 << 20
        tuned, _ = mc.mc_autotune(db.handle, cp, [mc.batch(int(w.qoffs[n_s]), d_reads, d_roffs, d_qoffs[: n_s + 1],
                                                           label, hits, top)], reps=1)
        mc.mc_db_set_tuning(db.handle, tuned)
        mc.mc_classify(db.handle, cp, w.n_seq, d_reads, d_roffs, nq, d_qoffs, label, hits, top)
        mc.mc_classify_status(db.handle)
        g_label, g_hits, g_top = host_u32(label), host_u32(hits), host_u32(top)

        # windows: closed form over the target lengths
        lens = np.diff(w.goffs).astype(np.int64)
        k, stride = w.db_params["k"], w.db_params["window_stride"]
        n_win = int(np.where(lens >= k, (lens - k + stride) // stride, 0).sum())
        assert st["n_windows"] == n_win

        # sample of queries and their features
        rng = np.random.default_rng(7)
        qs = np.sort(rng.choice(nq, size=2000, replace=False))
        mates = [(int(w.qoffs[q]), int(w.qoffs[q + 1])) for q in qs]
        sub_reads, sub_roffs, sub_qoffs = [], [0], [0]
        for a, b in mates:
            for i in range(a, b):
                sub_reads.append(w.reads[int(w.roffs[i]):int(w.roffs[i + 1])])
                sub_roffs.append(sub_roffs[-1] + int(w.roffs[i + 1] - w.roffs[i]))
            sub_qoffs.append(sub_qoffs[-1] + (b - a))
        sub_reads = np.concatenate(sub_reads)
        sub_roffs = np.array(sub_roffs, dtype=np.uint64)
        sub_qoffs = np.array(sub_qoffs, dtype=np.uint32)
        _, sk, cnt = oracle.sketch(sub_reads, sub_roffs, **w.db_params)
        feats = np.unique(np.concatenate([sk[i][:cnt[i]] for i in range(len(cnt))]))
        lo, hi = 0, (1 << 32) // 2048
        keys = np.unique(np.concatenate([feats, np.arange(lo, hi, dtype=np.uint32)]))

        odb = oracle.DB(w.genomes, w.goffs, key_filter=keys, n_threads=os.cpu_count() or 1, **w.db_params)
        ost = odb.stats()
        assert st["n_pairs"] == ost["n_pairs"]
        assert st["n_windows"] == ost["n_windows"]

        # database dump of the key range
        gk, gc, gl = db.dump(lo, hi)
        ok, oc, ol = odb.dump(lo, hi)
        assert len(gk) == len(ok) > 1000
        assert (gk == ok).all() and (gc == oc).all() and (gl == ol).all()

        # classification of the sampled queries
        ol_, oh_, ot_ = odb.classify(w.parent, w.taxon_of_target, sub_reads, sub_roffs, sub_qoffs,
                                     n_threads=os.cpu_count() or 1, **w.cls_params)
        assert (g_hits[qs] == oh_).all()
        assert (g_top[qs] == ot_).all()
        assert (g_label[qs] == ol_).all()
        # sanity: most reads from inserted genomes get their species or strain
        real = w.truth[qs] != synth.NO_GENOME
        assert (g_label[qs][real] != oracle.NO_TAXON).mean() > 0.9
    finally:
        db.free()
