"""Batched classification of mixed-length query batches: one launch set
over many batches (mc_classify_batches), CUDA-graph plans (mc_plan) and the
autotuner.  Every form must give, bit for bit, the results of one
mc_classify call per batch and of the oracle."""
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


@pytest.fixture(scope="module")
def setup(mc):
    w = synth.mid_workload(seed=31, n_pairs=10, n_families=1, genera_per_family=3, len_scale=0.03, held_genera=0)
    db = mc.Database.create(w.parent, **w.db_params)
    db.add_targets(dev(w.genomes), dev(w.goffs), w.taxon_of_target)
    db.finalize()
    sizes = [700, 0, 1, 2500, 37, 1200, 5, 900, 64, 333, 0, 1500]
    batches = synth.mixed_batches(9, w.genomes, w.goffs, sizes=sizes)
    yield w, db, batches
    db.free()


class DevBatch:
    """A batch on the device with its output tensors."""

    def __init__(self, mc, reads, roffs, qoffs):
        import torch
        self.nq = len(qoffs) - 1
        self.n_seq = len(roffs) - 1
        self.seq = dev(reads) if len(reads) else torch.zeros(1, dtype=torch.uint8, device="cuda")
        self.offs = dev(roffs)
        self.qoffs = dev(qoffs)
        n = max(1, self.nq)
        self.label = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        self.hits = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        self.top = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        self.desc = mc.batch(self.n_seq, self.seq, self.offs, self.qoffs, self.label, self.hits, self.top)

    def reset(self):
        for t in (self.label, self.hits, self.top):
            t.fill_(-7)

    def result(self):
        return [host_u32(t)[: self.nq] for t in (self.label, self.hits, self.top)]


def _per_batch(mc, db, cp, b: DevBatch):
    b.reset()
    if b.nq:
        mc.mc_classify(db.handle, cp, b.n_seq, b.seq, b.offs, b.nq, b.qoffs, b.label, b.hits, b.top)
    mc.mc_classify_status(db.handle)
    return b.result()


def _assert_same(xs, ys):
    for a, b in zip(xs, ys):
        assert len(a) == len(b) and (a == b).all()


def test_batches_match_per_batch_calls_and_oracle(mc, setup):
    w, db, batches = setup
    cp = mc.classify_params(**dict(w.cls_params, max_insert=0))
    dbs = [DevBatch(mc, *b[:3]) for b in batches]
    want = [_per_batch(mc, db, cp, b) for b in dbs]
    for b in dbs:
        b.reset()
    mc.mc_classify_batches(db.handle, cp, [b.desc for b in dbs])
    mc.mc_classify_status(db.handle)
    for b, r in zip(dbs, want):
        _assert_same(b.result(), r)
    # the oracle over all batches at once
    reads, roffs, qoffs, _ = synth.concat_batches(batches)
    odb = oracle.DB(w.genomes, w.goffs, **w.db_params)
    ol, oh, ot = odb.classify(w.parent, w.taxon_of_target, reads, roffs, qoffs, n_threads=8,
                              **dict(w.cls_params, max_insert=0))
    got = [np.concatenate([b.result()[i] for b in dbs]) for i in range(3)]
    _assert_same(got, [ol, oh, ot])


# score_mode 1 = sort path (the default for 32-bit locations), 2 = hash path;
# the expected results come from the default shape, so every hash-path shape
# is also checked against the sort path
TUNINGS = [
    dict(),
    dict(sort_max=256),
    dict(sort_max=512, probe_batch=8, lookup_warps=4),
    dict(score_mode=1, sort_max=1024, probe_batch=2),
    dict(score_mode=1, sort_max=2048, probe_batch=4),
    dict(score_mode=2),
    dict(score_mode=2, hist_slots=256, probe_batch=2, gather_batch=4, lookup_warps=4, score_warps=2),
    dict(score_mode=2, hist_slots=1024, probe_batch=8, gather_batch=16, lookup_warps=8, score_warps=4),
    dict(score_mode=2, hist_slots=256, gather_batch=16, score_warps=4),
    dict(wide_keys=1),
    dict(score_mode=2, hist_slots=256, probe_batch=2, gather_batch=4, score_warps=2, wide_keys=1),
]


@pytest.mark.parametrize("t", TUNINGS, ids=lambda t: "-".join(f"{k[:2]}{v}" for k, v in t.items()) or "default")
def test_every_tuning_gives_the_same_results(mc, setup, t):
    w, db, batches = setup
    cp = mc.classify_params(**dict(w.cls_params, max_insert=390))
    dbs = [DevBatch(mc, *b[:3]) for b in batches]
    want = [_per_batch(mc, db, cp, b) for b in dbs]
    for b in dbs:
        b.reset()
    mc.mc_classify_batches(db.handle, cp, [b.desc for b in dbs], mc.tuning(**t))
    mc.mc_classify_status(db.handle)
    for b, r in zip(dbs, want):
        _assert_same(b.result(), r)
    # the same tuning as the database default for plain calls
    mc.mc_db_set_tuning(db.handle, mc.tuning(**t))
    try:
        for b, r in zip(dbs, want):
            _assert_same(_per_batch(mc, db, cp, b), r)
    finally:
        mc.mc_db_set_tuning(db.handle, None)


def test_invalid_tuning_is_rejected(mc, setup):
    w, db, batches = setup
    for bad in [dict(hist_slots=300), dict(probe_batch=3), dict(gather_batch=32), dict(lookup_warps=16),
                dict(score_warps=8), dict(score_mode=3), dict(sort_max=300)]:
        with pytest.raises(mc.McError) as e:
            mc.mc_db_set_tuning(db.handle, mc.tuning(**bad))
        assert e.value.code == mc.MC_ERR_ARG


def test_plan_replays_new_batch_sets(mc, setup):
    w, db, batches = setup
    cp = mc.classify_params(**w.cls_params)
    dbs = [DevBatch(mc, *b[:3]) for b in batches]
    want = [_per_batch(mc, db, cp, b) for b in dbs]
    total = sum(b.nq for b in dbs)
    plan = mc.Plan(db.handle, cp, max_batches=len(dbs), max_queries=total)
    try:
        assert plan.kernels == 6  # lookup, sort-path size classes up to 1024 (default), medium path, large path
        for subset in [list(range(len(dbs))), [3, 0, 5], [7], list(range(len(dbs)))[::-1], []]:
            for b in dbs:
                b.reset()
            plan.run([dbs[i].desc for i in subset])
            mc.mc_classify_status(db.handle)
            for i in subset:
                _assert_same(dbs[i].result(), want[i])
            for i in set(range(len(dbs))) - set(subset):
                if dbs[i].nq:
                    assert (dbs[i].result()[0] == np.uint32(0xFFFFFFF9)).all()  # untouched
        with pytest.raises(mc.McError) as e:
            plan.run([dbs[0].desc] * (len(dbs) + 1))
        assert e.value.code == mc.MC_ERR_CAPACITY
    finally:
        plan.free()
    small = mc.Plan(db.handle, cp, max_batches=4, max_queries=100)
    try:
        with pytest.raises(mc.McError) as e:
            small.run([dbs[3].desc])
        assert e.value.code == mc.MC_ERR_CAPACITY
    finally:
        small.free()


def test_plan_recaptures_after_live_extension(mc):
    """A plan made before an extension serves the extended database."""
    w = synth.mid_workload(seed=41, n_pairs=10, n_families=1, genera_per_family=2, len_scale=0.02, held_genera=0)
    n = len(w.goffs) - 1
    half = n // 2
    cp = mc.classify_params(**w.cls_params)
    db = mc.Database.create(w.parent, **w.db_params)
    try:
        lo = int(w.goffs[half])
        db.add_targets(dev(w.genomes[:lo]), dev(w.goffs[: half + 1]), w.taxon_of_target[:half])
        db.finalize()
        batches = synth.mixed_batches(4, w.genomes, w.goffs, sizes=[400, 800, 50])
        dbs = [DevBatch(mc, *b[:3]) for b in batches]
        plan = mc.Plan(db.handle, cp, max_batches=3, max_queries=1250)
        try:
            plan.run([b.desc for b in dbs])
            before = [b.result() for b in dbs]
            db.add_targets(dev(w.genomes[lo:]), dev((w.goffs[half:] - np.uint64(lo)).astype(np.uint64)),
                           w.taxon_of_target[half:])
            db.finalize()
            for b in dbs:
                b.reset()
            plan.run([b.desc for b in dbs])
            mc.mc_classify_status(db.handle)
            after = [b.result() for b in dbs]
        finally:
            plan.free()
        reads, roffs, qoffs, _ = synth.concat_batches(batches)
        ol, oh, ot = oracle.DB(w.genomes, w.goffs, **w.db_params).classify(
            w.parent, w.taxon_of_target, reads, roffs, qoffs, n_threads=8, **w.cls_params)
        _assert_same([np.concatenate([a[i] for a in after]) for i in range(3)], [ol, oh, ot])
        # reads of the second half's genomes were unclassifiable or worse before
        assert sum(int((a[1] != b[1]).sum()) for a, b in zip(after, before)) > 0
    finally:
        db.free()


def test_autotune_picks_a_valid_setting_with_equal_results(mc, setup):
    w, db, batches = setup
    cp = mc.classify_params(**w.cls_params)
    dbs = [DevBatch(mc, *b[:3]) for b in batches]
    want = [_per_batch(mc, db, cp, b) for b in dbs]
    best, rec = mc.mc_autotune(db.handle, cp, [b.desc for b in dbs], reps=2)
    assert len(rec) == 6 + 18 + 4  # lookup shapes, hash-path shapes, sort-path size limits
    assert {r[0] for r in rec} == {0, 1} and all(r[2] > 0 for r in rec)
    bt = best.as_dict()
    assert bt["hist_slots"] in (256, 512, 1024) and bt["probe_batch"] in (2, 4, 8)
    for b in dbs:
        b.reset()
    mc.mc_classify_batches(db.handle, cp, [b.desc for b in dbs], best)
    mc.mc_classify_status(db.handle)
    for b, r in zip(dbs, want):
        _assert_same(b.result(), r)


def test_classify_in_flight_during_extension_sees_its_epoch(mc):
    """A classify enqueued on another stream before an extension reads the
    layout it was enqueued against, even though finalize replaces it."""
    import torch
    w = synth.mid_workload(seed=43, n_pairs=20000, n_families=1, genera_per_family=2, len_scale=0.02,
                           held_genera=0)
    n = len(w.goffs) - 1
    half = n // 2
    lo = int(w.goffs[half])
    cp = mc.classify_params(**w.cls_params)
    db = mc.Database.create(w.parent, **w.db_params)
    try:
        db.add_targets(dev(w.genomes[:lo]), dev(w.goffs[: half + 1]), w.taxon_of_target[:half])
        db.finalize()
        b = DevBatch(mc, w.reads, w.roffs, w.qoffs)
        want = _per_batch(mc, db, cp, b)
        b.reset()
        side = torch.cuda.Stream()
        for _ in range(3):  # keep the side stream busy while the database changes
            mc.mc_classify(db.handle, cp, b.n_seq, b.seq, b.offs, b.nq, b.qoffs, b.label, b.hits, b.top,
                           stream=side)
        db.add_targets(dev(w.genomes[lo:]), dev((w.goffs[half:] - np.uint64(lo)).astype(np.uint64)),
                       w.taxon_of_target[half:])
        db.finalize()
        side.synchronize()
        mc.mc_classify_status(db.handle, side)
        _assert_same(b.result(), want)
    finally:
        db.free()


def test_random_read_bandwidth_is_measured(mc):
    import membench
    membench.build()
    g16 = membench.random_read_gbs(1 << 30, 16, 1 << 24)
    g32 = membench.random_read_gbs(1 << 30, 32, 1 << 24)
    assert 10.0 < g16 < 20000.0 and 10.0 < g32 < 20000.0
    with pytest.raises(ValueError):
        membench.random_read_gbs(1 << 30, 24, 1 << 20)
