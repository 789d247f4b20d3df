"""Served classification (mc_server): jobs that arrive while others are on
the GPU are batched together, split across launch sets and admitted by
device memory; each job's result must be the same as when it is classified
alone, and after live extensions each job must match the oracle on the
database state (epoch) it was classified against."""
import threading
import time

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


def _alone(mc, db, cp, reads, roffs, qoffs):
    import torch
    nq = len(qoffs) - 1
    out = [torch.empty(max(1, nq), dtype=torch.int32, device="cuda") for _ in range(3)]
    if nq:
        mc.mc_classify(db.handle, cp, len(roffs) - 1, dev(reads) if len(reads) else dev(np.zeros(1, np.uint8)),
                       dev(roffs), nq, dev(qoffs), *out)
    mc.mc_classify_status(db.handle)
    return [host_u32(t)[:nq] for t in out]


def _host_job(job, pinned):
    """Host copies of a job's inputs and outputs (page-locked or pageable)."""
    import torch
    reads, roffs, qoffs = job[:3]
    nq = len(qoffs) - 1
    if pinned:
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        ins = [t(reads if len(reads) else np.zeros(1, np.uint8)), t(roffs.view(np.int64)), t(qoffs.view(np.int32))]
        outs = [torch.empty(max(1, nq), dtype=torch.int32).pin_memory() for _ in range(3)]
        view = lambda x: x.numpy().view(np.uint32)[:nq]
    else:
        ins = [np.ascontiguousarray(reads if len(reads) else np.zeros(1, np.uint8)), roffs, qoffs]
        outs = [np.zeros(max(1, nq), np.uint32) for _ in range(3)]
        view = lambda x: x[:nq]
    return ins, outs, (lambda: [view(o) for o in outs])


def test_results_are_the_same_alone_and_in_the_mix(mc):
    w = synth.mid_workload(seed=51, n_pairs=10, n_families=1, genera_per_family=3, len_scale=0.03, held_genera=0)
    db = mc.Database.create(w.parent, **w.db_params)
    db.add_targets(dev(w.genomes), dev(w.goffs), w.taxon_of_target)
    db.finalize()
    cp = mc.classify_params(**dict(w.cls_params, max_insert=0))
    rng = np.random.default_rng(3)
    sizes = np.clip(np.exp(rng.normal(np.log(800), 1.2, 40)).astype(int), 1, 9000)
    sizes[5] = 0
    jobs = synth.mixed_batches(61, w.genomes, w.goffs, sizes=sizes, len_lo=75, len_hi=250)
    want = [_alone(mc, db, cp, *j[:3]) for j in jobs]
    srv = mc.Server(db.handle, cp, n_streams=3, max_set_queries=3000, max_set_jobs=7)
    try:
        host = [_host_job(j, pinned=(i % 2 == 0)) for i, j in enumerate(jobs)]
        ids = [None] * len(jobs)

        def submitter(lo, hi):
            for i in range(lo, hi):
                ins, outs, _ = host[i]
                ids[i] = srv.submit(len(jobs[i][1]) - 1, *ins, *outs)
                time.sleep(0.0005 * (i % 3))

        ths = [threading.Thread(target=submitter, args=(a, a + 10)) for a in range(0, 40, 10)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        infos = [srv.wait(i, timeout=120.0) for i in ids]
        assert all(x is not None and x["status"] == 0 for x in infos)
        for (ins, outs, get), wnt, n in zip(host, want, sizes):
            got = get()
            for a, b in zip(got, wnt):
                assert (a == b).all()
        st = srv.stats()
        assert st["jobs_done"] == 40 and st["queries_done"] == int(sizes.sum())
        assert st["launch_sets"] >= int(np.ceil(sizes.sum() / 3000))
        assert 0 < st["p50_latency_s"] <= st["p99_latency_s"] <= st["max_latency_s"]
        assert max(x["pieces"] for x in infos) >= 3  # the largest jobs were split
        assert st["hbm_in_use"] == 0
    finally:
        srv.free()
        db.free()


def test_live_extension_epochs_match_the_oracle(mc):
    w = synth.mid_workload(seed=53, n_pairs=10, n_families=1, genera_per_family=2, len_scale=0.02, held_genera=0)
    n = len(w.goffs) - 1
    cuts = [n // 2, 3 * n // 4, n]
    cp = mc.classify_params(**dict(w.cls_params, max_insert=0))
    db = mc.Database.create(w.parent, **w.db_params)
    db.add_targets(dev(w.genomes[: int(w.goffs[cuts[0]])]), dev(w.goffs[: cuts[0] + 1]), w.taxon_of_target[:cuts[0]])
    db.finalize()
    jobs = synth.mixed_batches(71, w.genomes, w.goffs, sizes=[300, 1200, 40, 700, 2500, 90, 800, 1500, 10, 600],
                               len_lo=75, len_hi=250)
    srv = mc.Server(db.handle, cp, n_streams=2, max_set_queries=1000)
    try:
        host = [_host_job(j, pinned=True) for j in jobs]
        sub = lambda i: srv.submit(len(jobs[i][1]) - 1, *host[i][0], *host[i][1])
        ids = [sub(i) for i in range(3)]
        srv.drain(120.0)
        for e, (a, b) in enumerate(zip(cuts[:-1], cuts[1:])):
            lo, hi = int(w.goffs[a]), int(w.goffs[b])
            ids += [sub(i) for i in range(3 + 2 * e, 5 + 2 * e)]
            first = srv.extend(w.genomes[lo:hi], w.goffs[a:b + 1] - np.uint64(lo), w.taxon_of_target[a:b])
            assert first == a
        ids += [sub(i) for i in range(7, 10)]
        infos = [srv.wait(i, timeout=120.0) for i in ids]
        st = srv.stats()
        assert st["extensions"] == 2 and st["epoch"] == 2
    finally:
        srv.free()
    try:
        assert [x["epoch"] for x in infos[:3]] == [0, 0, 0]
        assert [x["epoch"] for x in infos[7:]] == [2, 2, 2]
        odbs = {}
        for i, x in enumerate(infos):
            e = x["epoch"]
            if e not in odbs:
                k = cuts[e]
                odbs[e] = oracle.DB(w.genomes[: int(w.goffs[k])], w.goffs[: k + 1], **w.db_params)
            want = odbs[e].classify(w.parent, w.taxon_of_target[: cuts[e]], *jobs[i][:3], n_threads=8,
                                    **dict(w.cls_params, max_insert=0))
            for a, b in zip(host[i][2]()[:3], want):
                assert (a == b).all(), (i, e)
        # the database the server left behind is the final state
        st = db.stats()
        assert st["n_targets"] == n and st["finalized"] == 1
    finally:
        db.free()


def test_admission_keeps_within_the_memory_limit(mc):
    w = synth.mid_workload(seed=55, n_pairs=10, n_families=1, genera_per_family=1, len_scale=0.02, held_genera=0)
    db = mc.Database.create(w.parent, **w.db_params)
    db.add_targets(dev(w.genomes), dev(w.goffs), w.taxon_of_target)
    db.finalize()
    cp = mc.classify_params(**w.cls_params)
    jobs = synth.mixed_batches(81, w.genomes, w.goffs, sizes=[2000] * 12, len_lo=75, len_hi=250)
    want = [_alone(mc, db, cp, *j[:3]) for j in jobs]
    limit = 3 << 20  # room for about two jobs at a time
    srv = mc.Server(db.handle, cp, n_streams=2, hbm_limit=limit)
    try:
        host = [_host_job(j, pinned=True) for j in jobs]
        ids = [srv.submit(len(j[1]) - 1, *h[0], *h[1]) for j, h in zip(jobs, host)]
        for i in ids:
            assert srv.wait(i, 120.0)["status"] == 0
        st = srv.stats()
        assert 0 < st["hbm_peak"] <= limit
        for h, wnt in zip(host, want):
            for a, b in zip(h[2](), wnt):
                assert (a == b).all()
        big = synth.mixed_batches(82, w.genomes, w.goffs, sizes=[40000], len_lo=250, len_hi=250)[0]
        hb = _host_job(big, pinned=False)
        with pytest.raises(mc.McError) as e:
            srv.submit(len(big[1]) - 1, *hb[0], *hb[1])
        assert e.value.code == mc.MC_ERR_OOM
        bad_q = jobs[0][2].copy()
        bad_q[-1] = len(jobs[0][1])  # one past the last mate
        with pytest.raises(mc.McError) as e:
            srv.submit(len(jobs[0][1]) - 1, host[0][0][0], host[0][0][1], bad_q, *host[0][1])
        assert e.value.code == mc.MC_ERR_ARG
    finally:
        srv.free()
        db.free()
