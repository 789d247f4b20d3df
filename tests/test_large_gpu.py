"""The large-database recipe: genera of bacterial-like genomes plus
repeat-rich eukaryote-like genomes whose repeated segments overfill buckets
(bucket cap, overflow counts).  A reduced instance is checked against the
oracle in full.  The full-size instance (10,000 genomes, about 14.3 Gbp,
50M read pairs) is built and classified in the launch configuration
bench.py times, and checked against the oracle on sampled outputs: the
oracle builds the buckets of every feature of 2,000 sampled queries (a
quarter of them from the repeat-rich genomes) plus every feature of one key
range, which are then complete, so the dump of that key range and the
labels, hit counts and top targets of the sampled queries must be equal.
Mixed-length query batches (sizes lognormal, lengths 50-300, single-end
and pairs) are classified against the same full-size database through a
CUDA-graph plan and checked the same way on 1,000 sampled queries."""
import os

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


def _sub_queries(w, qs):
    """Reads, read offsets and query offsets of the queries qs of w."""
    sub_reads, sub_roffs, sub_qoffs = [], [0], [0]
    for q in qs:
        a, b = int(w.qoffs[q]), int(w.qoffs[q + 1])
        for i in range(a, b):
            sub_reads.append(w.reads[int(w.roffs[i]):int(w.roffs[i + 1])])
            sub_roffs.append(sub_roffs[-1] + int(w.roffs[i + 1] - w.roffs[i]))
        sub_qoffs.append(sub_qoffs[-1] + (b - a))
    return (np.concatenate(sub_reads), np.array(sub_roffs, dtype=np.uint64), np.array(sub_qoffs, dtype=np.uint32))


def test_fullsize_large_database_matches_oracle_on_samples(mc):
    import torch
    w = synth.large_workload(seed=1002, scaled=True)
    p = w.db_params
    n_threads = os.cpu_count() or 1
    db = mc.Database.create(w.parent, **p)
    try:
        db.add_targets(dev(w.genomes), dev(w.goffs), w.taxon_of_target)
        db.finalize()
        st = db.stats()
        lens = np.diff(w.goffs).astype(np.int64)
        k, stride = p["k"], p["window_stride"]
        assert st["n_windows"] == int(np.where(lens >= k, (lens - k + stride) // stride, 0).sum())
        assert st["overflow_keys"] > 0 and st["n_locations"] + st["dropped_locations"] == st["n_pairs"]
        assert 0 < st["load_factor"] <= 0.5

        # every pair classified in one call, with the autotuner's launch shape (as the bench does)
        nq = w.n_queries
        label = torch.empty(nq, dtype=torch.int32, device="cuda")
        hits = torch.empty(nq, dtype=torch.int32, device="cuda")
        top = torch.empty(nq, dtype=torch.int32, device="cuda")
        cp = mc.classify_params(**w.cls_params)
        d_reads, d_roffs, d_qoffs = dev(w.reads), dev(w.roffs), dev(w.qoffs)
        n_s = 1 << 20
        tuned, _ = mc.mc_autotune(db.handle, cp, [mc.batch(int(w.qoffs[n_s]), d_reads, d_roffs, d_qoffs[: n_s + 1],
                                                           label, hits, top)], reps=1)
        mc.mc_db_set_tuning(db.handle, tuned)
        mc.mc_classify(db.handle, cp, w.n_seq, d_reads, d_roffs, nq, d_qoffs, label, hits, top)
        mc.mc_classify_status(db.handle)
        g_label, g_hits, g_top = host_u32(label), host_u32(hits), host_u32(top)
        del d_reads, d_roffs, d_qoffs, label, hits, top

        # sampled queries: uniform ones plus queries from the repeat-rich genomes
        rng = np.random.default_rng(11)
        n_bact = len(w.taxon_of_target) - 200
        euk = np.nonzero((w.truth >= n_bact) & (w.truth != synth.NO_GENOME))[0]
        qs = np.unique(np.concatenate([rng.choice(nq, size=1500, replace=False),
                                       rng.choice(euk, size=500, replace=False)]))
        sub_reads, sub_roffs, sub_qoffs = _sub_queries(w, qs)
        _, sk, cnt = oracle.sketch(sub_reads, sub_roffs, **p)
        feats = np.unique(np.concatenate([sk[i][:cnt[i]] for i in range(len(cnt))]))

        # mixed-length batches against the same database (the batched workload:
        # sizes lognormal, lengths 50-300, half single-end half pairs), run as
        # one replay of a CUDA-graph plan with the tuned shape; 1,000 sampled
        # queries of them are checked below
        batches = synth.mixed_batches(1003, w.genomes, w.goffs, n_batches=24)
        mb = [(dev(r) if len(r) else dev(np.zeros(1, np.uint8)), dev(ro), dev(qo), len(ro) - 1, len(qo) - 1)
              for r, ro, qo, _ in batches]
        outs = [[torch.empty(max(1, nqb), dtype=torch.int32, device="cuda") for _ in range(3)]
                for *_, nqb in mb]
        descs = [mc.batch(n_seq, r, ro, qo, *o) for (r, ro, qo, n_seq, _), o in zip(mb, outs)]
        cp0 = mc.classify_params(**dict(w.cls_params, max_insert=0))
        plan = mc.Plan(db.handle, cp0, len(descs), sum(x[4] for x in mb), tuned)
        try:
            plan.run(descs)
            mc.mc_classify_status(db.handle)
        finally:
            plan.free()
        all_r, all_ro, all_qo, _ = synth.concat_batches(batches)
        got_b = [np.concatenate([host_u32(o[i])[: x[4]] for o, x in zip(outs, mb)]) for i in range(3)]
        nb = len(all_qo) - 1

        class _W:  # the concatenated batches, shaped for _sub_queries
            reads, roffs, qoffs = all_r, all_ro, all_qo
        qb = np.sort(rng.choice(nb, size=1000, replace=False))
        b_reads, b_roffs, b_qoffs = _sub_queries(_W, qb)
        _, skb, cntb = oracle.sketch(b_reads, b_roffs, **p)
        feats = np.unique(np.concatenate([feats] + [skb[i][:cntb[i]] for i in range(len(cntb))]))
        lo, hi = 0, (1 << 32) // 4096
        keys = np.unique(np.concatenate([feats, np.arange(lo, hi, dtype=np.uint32)]))
        odb = oracle.DB(w.genomes, w.goffs, key_filter=keys, n_threads=n_threads, **p)
        ost = odb.stats()
        assert st["n_pairs"] == ost["n_pairs"] and st["n_windows"] == ost["n_windows"]

        # database dump of the key range, including overflowing buckets
        gk, gc, gl = db.dump(lo, hi)
        ok, oc, ol = odb.dump(lo, hi)
        assert len(gk) == len(ok) > 1000
        assert (gk == ok).all() and (gc == oc).all() and (gl == ol).all()
        assert (gc == p["bucket_cap"]).any()

        # classification of the sampled queries
        ol_, oh_, ot_ = odb.classify(w.parent, w.taxon_of_target, sub_reads, sub_roffs, sub_qoffs,
                                     n_threads=n_threads, **w.cls_params)
        assert (g_hits[qs] == oh_).all()
        assert (g_top[qs] == ot_).all()
        assert (g_label[qs] == ol_).all()
        assert (g_label[qs] != oracle.NO_TAXON).mean() > 0.8
        # the sampled queries of the mixed batches
        bl, bh, bt = odb.classify(w.parent, w.taxon_of_target, b_reads, b_roffs, b_qoffs, n_threads=n_threads,
                                  **dict(w.cls_params, max_insert=0))
        assert (got_b[1][qb] == bh).all()
        assert (got_b[2][qb] == bt).all()
        assert (got_b[0][qb] == bl).all()
    finally:
        db.free()
