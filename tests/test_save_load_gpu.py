"""A database written by mc_db_save and read back by mc_db_load (the
condensed layout of Section 4.2, stored after the build of Section 4.1) is
the same database: equal dump, counters and classification, bit for bit, and
it can be extended like the one it was saved from."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import dev, gpu_build, gpu_classify

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2106_08150_gb300 import mc as m
    m.use_torch_allocator()
    return m


def _dump_equal(a, b):
    for x, y in zip(a, b):
        assert len(x) == len(y) and (x == y).all()


def test_save_load_roundtrip(mc, tmp_path):
    w = synth.tiny_workload()
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    path = str(tmp_path / "tiny.mcdb")
    db.save(path)
    db2 = mc.Database.load(path)
    try:
        st, st2 = db.stats(), db2.stats()
        for k in ["n_targets", "n_windows", "n_pairs", "n_keys", "n_locations", "overflow_keys", "table_slots",
                  "max_probe", "finalized", "max_depth"]:
            assert st[k] == st2[k], k
        _dump_equal(db.dump(), db2.dump())
        cp = {k: v for k, v in w.cls_params.items() if k != "max_candidates"}
        a = gpu_classify(mc, db, w.reads, w.roffs, w.qoffs, with_cands=True, **cp)
        b = gpu_classify(mc, db2, w.reads, w.roffs, w.qoffs, with_cands=True, **cp)
        for x, y in zip(a, b):
            assert (x == y).all()
        want = oracle.DB(w.genomes, w.goffs, **w.db_params).classify(
            w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, max_candidates=4, **cp)
        for x, y in zip(b[:3], want):
            assert (x == y).all()
    finally:
        db.free()
        db2.free()


def test_loaded_database_extends_like_a_fresh_build(mc, tmp_path):
    w = synth.mid_workload(seed=12, n_pairs=10, n_families=1, genera_per_family=2, len_scale=0.01, held_genera=0)
    p = dict(w.db_params, bucket_cap=4)
    n = len(w.goffs) - 1
    half = n // 2
    db = gpu_build(mc, w.genomes[: int(w.goffs[half])], w.goffs[: half + 1], w.parent, w.taxon_of_target[:half], **p)
    path = str(tmp_path / "half.mcdb")
    db.save(path)
    db.free()
    db2 = mc.Database.load(path)
    try:
        lo, hi = int(w.goffs[half]), int(w.goffs[n])
        first = db2.add_targets(dev(w.genomes[lo:hi]), dev((w.goffs[half:] - np.uint64(lo)).astype(np.uint64)),
                                w.taxon_of_target[half:])
        assert first == half
        db2.finalize()
        odb = oracle.DB(w.genomes, w.goffs, **p)
        _dump_equal(db2.dump(), odb.dump())
        ost, st = odb.stats(), db2.stats()
        # overflow_keys is not compared: a re-finalize sees only the kept
        # locations of earlier targets (as in any live extension)
        for k in ["n_targets", "n_windows", "n_pairs", "n_keys"]:
            assert st[k] == ost[k], k
        assert st["n_locations"] == ost["n_locations"]
    finally:
        db2.free()


def test_save_before_finalize_is_a_state_error(mc, tmp_path):
    w = synth.tiny_workload()
    db = mc.Database.create(w.parent, **w.db_params)
    try:
        with pytest.raises(mc.McError) as e:
            db.save(str(tmp_path / "x.mcdb"))
        assert e.value.code == mc.MC_ERR_STATE
    finally:
        db.free()


def test_truncated_file_is_rejected(mc, tmp_path):
    w = synth.tiny_workload()
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    path = tmp_path / "t.mcdb"
    db.save(str(path))
    db.free()
    data = path.read_bytes()
    cut = tmp_path / "cut.mcdb"
    cut.write_bytes(data[: len(data) - 100])
    with pytest.raises(mc.McError) as e:
        mc.Database.load(str(cut))
    assert e.value.code == mc.MC_ERR_ARG
