"""Partitioned databases on the GPU (Sections 4.2 and 4.3), three shards on
one device in the order the protocol of paper_2106_08150_gb300.shard runs
them (feature counts of every shard, then each shard finalized against the
earlier shards' counts, then every shard's top-m lists merged).  The shards'
buckets together, and the merged labels, hit counts, top targets and top-m
lists, must equal the single-database oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import dev, host_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2106_08150_gb300 import mc as m
    m.use_torch_allocator()
    return m


def _workload(cap):
    w = synth.mid_workload(seed=31, n_pairs=1500, n_families=1, genera_per_family=3, len_scale=0.02,
                           held_genera=0)
    w.db_params = dict(w.db_params, bucket_cap=cap)
    return w


def _shards(mc, w, world):
    from paper_2106_08150_gb300.shard import GpuShard, shard_ranges
    tg = dev(w.taxon_of_target)
    out = []
    for lo, hi in shard_ranges(w.goffs, world):
        a, b = int(w.goffs[lo]), int(w.goffs[hi])
        out.append(GpuShard(mc, w.parent, lo, dev(w.genomes[a:b]), dev((w.goffs[lo:hi + 1] - np.uint64(a))),
                            w.taxon_of_target[lo:hi], tg, **w.db_params))
    return out


@pytest.mark.parametrize("cap,world", [(6, 3), (254, 2), (2, 4)])
def test_sharded_database_and_merged_classification_equal_the_single_oracle(mc, cap, world):
    w = _workload(cap)
    shards = _shards(mc, w, world)
    try:
        counts = [s.feature_counts() for s in shards]
        for r, s in enumerate(shards):
            s.finalize_after(counts[:r])
        whole = oracle.DB(w.genomes, w.goffs, **w.db_params)
        # buckets: the shards' buckets of a feature, in shard order (global ids), are the single bucket
        buckets = {}
        for s in shards:
            k, c, l = s.db.dump()
            l = l + (np.uint64(s.merge_base) << np.uint64(32))
            off = 0
            for key, cnt in zip(k, c):
                buckets.setdefault(int(key), []).extend(l[off:off + cnt].tolist())
                off += int(cnt)
        wk, wc, wl = whole.dump()
        assert sorted(buckets) == wk.tolist()
        off = 0
        for key, cnt in zip(wk, wc):
            assert buckets[int(key)] == wl[off:off + cnt].tolist()
            off += int(cnt)
        st = [s.db.stats() for s in shards]
        ost = whole.stats()
        assert sum(x["n_locations"] for x in st) == ost["n_locations"]
        assert sum(x["n_pairs"] for x in st) == ost["n_pairs"]
        # merged classification
        cp = dict(w.cls_params, max_candidates=4)
        d_r, d_ro, d_qo = dev(w.reads), dev(w.roffs), dev(w.qoffs)
        lists = [s.classify_cands(d_r, d_ro, d_qo, **cp) for s in shards]
        label, hits, top, cands = shards[0].merge(lists, [s.merge_base for s in shards], **cp)
        want = whole.classify(w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, with_cands=True, **cp)
        assert (host_u32(hits) == want[1]).all()
        assert (host_u32(top) == want[2]).all()
        assert (host_u32(cands).reshape(want[-1].shape) == want[-1]).all()
        assert (host_u32(label) == want[0]).all()
    finally:
        for s in shards:
            s.free()


def test_feature_counts_capacity_and_state(mc):
    w = _workload(6)
    s = _shards(mc, w, 1)[0]
    try:
        n = mc.mc_db_feature_counts(s.db.handle)
        assert n > 100
        import torch
        small = torch.empty(10, dtype=torch.int32, device="cuda")
        with pytest.raises(mc.McError) as e:
            mc.mc_db_feature_counts(s.db.handle, small, small, 10)
        assert e.value.code == mc.MC_ERR_CAPACITY
        keys, counts = s.feature_counts()
        k = host_u32(keys)
        assert (np.diff(k.astype(np.int64)) > 0).all()  # ascending, distinct
        c = host_u32(counts)
        assert c.min() >= 1 and c.max() <= 6
        s.finalize_after([])
        with pytest.raises(mc.McError) as e:
            mc.mc_db_feature_counts(s.db.handle)
        assert e.value.code == mc.MC_ERR_STATE
        # a shard finalized without prior is the plain database
        odb = oracle.DB(w.genomes, w.goffs, **w.db_params)
        gk, gc, gl = s.db.dump()
        ok, oc, ol = odb.dump()
        assert (gk == ok).all() and (gc == oc).all() and (gl == ol).all()
    finally:
        s.free()


def test_saved_and_loaded_shards_merge_to_the_single_oracle(mc, tmp_path):
    """Partitions saved one file per shard and loaded again (Section 4.3)
    classify and merge exactly like the single database."""
    from paper_2106_08150_gb300.shard import GpuShard
    w = _workload(6)
    shards = _shards(mc, w, 3)
    try:
        counts = [s.feature_counts() for s in shards]
        for r, s in enumerate(shards):
            s.finalize_after(counts[:r])
        for r, s in enumerate(shards):
            s.save(str(tmp_path / f"shard{r}.mcdb"))
    finally:
        for s in shards:
            s.free()
    tg = dev(w.taxon_of_target)
    loaded = [GpuShard.load(mc, str(tmp_path / f"shard{r}.mcdb"), tg) for r in range(3)]
    try:
        cp = dict(w.cls_params, max_candidates=4)
        d_r, d_ro, d_qo = dev(w.reads), dev(w.roffs), dev(w.qoffs)
        lists = [s.classify_cands(d_r, d_ro, d_qo, **cp) for s in loaded]
        label, hits, top, cands = loaded[0].merge(lists, [s.merge_base for s in loaded], **cp)
        whole = oracle.DB(w.genomes, w.goffs, **w.db_params)
        want = whole.classify(w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, with_cands=True, **cp)
        assert [s.merge_base for s in loaded] == sorted(s.merge_base for s in loaded)
        assert (host_u32(label) == want[0]).all()
        assert (host_u32(hits) == want[1]).all()
        assert (host_u32(top) == want[2]).all()
        assert (host_u32(cands).reshape(want[-1].shape) == want[-1]).all()
    finally:
        for s in loaded:
            s.free()
