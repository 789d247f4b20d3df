"""Partitioned databases on CPU (Sections 4.2 and 4.3).

1. The oracle's shard rule against the plain oracle: three shards of
   contiguous target ranges, each keeping at most cap - prior(f) locations
   of feature f (prior = the earlier shards' counts), hold together exactly
   the single database (same buckets), and merging their top-m lists gives
   the single database's labels, hits, top targets and top-m lists.
2. The exchange protocol of paper_2106_08150_gb300.shard over gloo ranks
   (world size 2 and 3), each rank running an oracle shard: the merged
   result on every rank equals the single-database oracle.
"""
import multiprocessing as mp
import os
import sys

import numpy as np
import pytest

import oracle
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _workload():
    # small genera with a low cap, so that many buckets are cut and the
    # prior counts decide what a later shard keeps
    w = synth.mid_workload(seed=31, n_pairs=1500, n_families=1, genera_per_family=3, len_scale=0.02,
                           held_genera=0)
    w.db_params = dict(w.db_params, bucket_cap=6)
    return w


def _merged_prior(prior):
    if not prior:
        return None
    keys = np.concatenate([np.asarray(k, dtype=np.uint32) for k, _ in prior])
    counts = np.concatenate([np.asarray(c, dtype=np.uint32) for _, c in prior])
    uk, inv = np.unique(keys, return_inverse=True)
    return uk, np.bincount(inv, weights=counts).astype(np.uint32)


class OracleShard:
    """A shard with the oracle as its engine (targets [lo, hi), global ids)."""

    def __init__(self, w, lo, hi):
        self.w, self.lo, self.hi = w, lo, hi
        a, b = int(w.goffs[lo]), int(w.goffs[hi])
        self.seq = w.genomes[a:b]
        self.offs = (w.goffs[lo:hi + 1] - np.uint64(a)).astype(np.uint64)
        self.merge_base = 0  # the oracle's locations carry global ids already
        self.pre = oracle.DB(self.seq, self.offs, target_base=lo, **w.db_params)
        self.db = None

    def feature_counts(self):
        import torch
        k, c = self.pre.feature_counts()
        return torch.from_numpy(k.view(np.int32).copy()), torch.from_numpy(c.view(np.int32).copy())

    def finalize_after(self, prior):
        pr = _merged_prior([(k.numpy().view(np.uint32), c.numpy().view(np.uint32)) for k, c in prior])
        self.db = oracle.DB(self.seq, self.offs, target_base=self.lo, prior=pr, **self.w.db_params)

    def classify_cands(self, reads, roffs, qoffs, *, max_candidates, **cp):
        import torch
        w = self.w
        out = self.db.classify(w.parent, w.taxon_of_target, reads, roffs, qoffs, max_candidates=max_candidates,
                               with_cands=True, **cp)
        return torch.from_numpy(out[-1].view(np.int32).reshape(-1).copy())

    def merge(self, lists, bases, *, max_candidates, **cp):
        m = max_candidates
        arrs = []
        for l, b in zip(lists, bases):
            a = l.numpy().view(np.uint32).reshape(-1, m, 4).copy()
            a[:, :, 1] += np.where(a[:, :, 0] > 0, np.uint32(b), np.uint32(0))
            arrs.append(a)
        return oracle.merge(arrs, self.w.parent, self.w.taxon_of_target, max_candidates=m, **cp)


def test_shard_ranges_are_contiguous_and_cover_all_targets():
    sys.path.insert(0, ROOT)
    from paper_2106_08150_gb300 import shard
    goffs = np.concatenate([[0], np.cumsum(np.arange(1, 41) * 1000)]).astype(np.uint64)
    for world in (1, 2, 3, 7, 40):
        r = shard.shard_ranges(goffs, world)
        assert r[0][0] == 0 and r[-1][1] == 40 and len(r) == world
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert all(hi > lo for lo, hi in r)


def test_oracle_shards_equal_the_single_database():
    w = _workload()
    p = w.db_params
    cp = dict(w.cls_params, max_candidates=4)
    n = w.n_targets
    cuts = [0, n // 3, (2 * n) // 3, n]
    whole = oracle.DB(w.genomes, w.goffs, **p)
    shards, counts = [], []
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        s = OracleShard(w, lo, hi)
        pr = _merged_prior(counts)
        s.db = oracle.DB(s.seq, s.offs, target_base=lo, prior=pr, **p)
        counts.append(s.pre.feature_counts())
        shards.append(s)
    # buckets: the shards' buckets of a feature, in shard order, are the single database's bucket
    wk, wc, wl = whole.dump()
    parts = [s.db.dump() for s in shards]
    buckets = {}
    for k, c, l in parts:
        off = 0
        for key, cnt in zip(k, c):
            buckets.setdefault(int(key), []).extend(l[off:off + cnt].tolist())
            off += cnt
    assert sorted(buckets) == wk.tolist()
    off = 0
    for key, cnt in zip(wk, wc):
        assert buckets[int(key)] == wl[off:off + cnt].tolist()
        off += cnt
    assert whole.stats()["overflow_keys"] > 50  # the cap cut many buckets
    # merged classification
    lists = [s.db.classify(w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, with_cands=True, **cp)[-1]
             for s in shards]
    got = oracle.merge(lists, w.parent, w.taxon_of_target, **cp)
    want = whole.classify(w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, with_cands=True, **cp)
    for a, b in zip(got, (want[0], want[1], want[2], want[-1])):
        assert (np.asarray(a) == np.asarray(b)).all()


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2106_08150_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = _workload()
        lo, hi = shard.shard_ranges(w.goffs, world)[rank]
        s = OracleShard(w, lo, hi)
        shard.build_partitioned(s)
        out = shard.classify_partitioned(s, w.reads, w.roffs, w.qoffs, **dict(w.cls_params, max_candidates=4))
        q.put((rank, [np.asarray(x) for x in out]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_protocol_over_gloo_ranks_matches_the_single_database(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + os.getpid() % 300 + 7 * world
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    w = _workload()
    cp = dict(w.cls_params, max_candidates=4)
    whole = oracle.DB(w.genomes, w.goffs, **w.db_params)
    want = whole.classify(w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, with_cands=True, **cp)
    want = (want[0], want[1], want[2], want[-1])
    for r in range(world):
        for a, b in zip(res[r], want):
            assert (np.asarray(a) == np.asarray(b)).all()
    assert (want[0] != oracle.NO_TAXON).mean() > 0.5
