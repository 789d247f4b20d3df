"""CUDA path (through the C ABI) against the CPU oracle, element by element.

Integer work throughout, so the bar is bit-exact equality: sketches, the
canonical database dump (features, sorted capped buckets), database
counters, and per-query labels, hit counts, top targets and top-m
candidate lists."""
import random

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import dev, gpu_build, gpu_classify, gpu_sketch, host_u32, offsets, u8

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2106_08150_gb300 import mc as m
    m.use_torch_allocator()
    return m


def _rand_seq(rng, n, n_rate=0.0, lower=0.0, alphabet="ACGT"):
    out = []
    for _ in range(n):
        c = rng.choice(alphabet)
        r = rng.random()
        if r < n_rate:
            c = rng.choice("NnRYX-")
        elif r < n_rate + lower:
            c = c.lower()
        out.append(c)
    return "".join(out)


def _oracle_db(seq, goffs, p):
    return oracle.DB(seq, goffs, **p)


def _assert_dump_equal(mc, db, odb):
    gk, gc, gl = db.dump()
    ok, oc, ol = odb.dump()
    assert len(gk) == len(ok)
    assert (gk == ok).all()
    assert (gc == oc).all()
    assert (gl == ol).all()


def _assert_stats_equal(db, odb):
    st, ost = db.stats(), odb.stats()
    for k in ["n_targets", "n_windows", "n_pairs", "n_keys", "n_locations", "overflow_keys"]:
        g = st["n_locations"] if k == "n_locations" else st[k]
        assert g == ost[k], (k, g, ost[k])


# ------------------------------------------------------------------ sketch
SKETCH_PARAMS = [
    dict(k=16, sketch_size=16, window_len=128, window_stride=113),
    dict(k=16, sketch_size=16, window_len=127, window_stride=112),
    dict(k=16, sketch_size=32, window_len=128, window_stride=50),
    dict(k=1, sketch_size=4, window_len=16, window_stride=3),
    dict(k=4, sketch_size=2, window_len=8, window_stride=5),
    dict(k=11, sketch_size=7, window_len=200, window_stride=190),
    dict(k=15, sketch_size=16, window_len=256, window_stride=242),
    dict(k=16, sketch_size=9, window_len=512, window_stride=497),
    dict(k=16, sketch_size=1, window_len=300, window_stride=1),
]


@pytest.mark.parametrize("p", SKETCH_PARAMS, ids=lambda p: f"k{p['k']}s{p['sketch_size']}w{p['window_len']}")
def test_sketch_matches_oracle(mc, p):
    rng = random.Random(p["k"] * 31 + p["window_len"])
    lens = [0, 1, p["k"] - 1, p["k"], p["k"] + 1, p["window_len"], p["window_len"] + 1, 3 * p["window_len"] + 7]
    lens += [rng.randint(0, 2000) for _ in range(30)]
    seqs = [_rand_seq(rng, L, n_rate=[0, 0.01, 0.2][i % 3], lower=0.1 * (i % 2)) for i, L in enumerate(lens)]
    seqs.append("ACGT" * 300)  # periodic: few distinct k-mers
    seqs.append("A" * 700)
    seq = "".join(seqs)
    offs = offsets([len(s) for s in seqs])
    win, sk, cnt = gpu_sketch(mc, seq, offs, **p)
    owin, osk, ocnt = oracle.sketch(seq, offs, **p)
    assert (win == owin).all()
    assert (cnt == ocnt).all()
    assert (sk == osk).all()


def test_sketch_full_tiny_genomes(mc):
    w = synth.tiny_workload(n_reads=10, n_decoys=1)
    win, sk, cnt = gpu_sketch(mc, w.genomes, w.goffs, **{k: w.db_params[k] for k in
                                                        ["k", "sketch_size", "window_len", "window_stride"]})
    owin, osk, ocnt = oracle.sketch(w.genomes, w.goffs, **w.db_params)
    assert len(cnt) == len(ocnt) > 14000
    assert (sk == osk).all() and (cnt == ocnt).all()


# ------------------------------------------------------------------- build
@pytest.fixture(scope="module")
def tiny():
    return synth.tiny_workload()


def test_build_dump_and_stats_tiny(mc, tiny):
    w = tiny
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    odb = _oracle_db(w.genomes, w.goffs, w.db_params)
    _assert_dump_equal(mc, db, odb)
    _assert_stats_equal(db, odb)
    st = db.stats()
    assert st["finalized"] == 1 and 0 < st["load_factor"] <= 0.5
    db.free()


def test_build_in_several_calls_and_with_empty_targets(mc):
    rng = random.Random(4)
    seqs = [_rand_seq(rng, rng.randint(0, 5000), n_rate=0.005) for _ in range(23)]
    seqs[3] = ""
    seqs[7] = "ACG"
    seq = "".join(seqs)
    goffs = offsets([len(s) for s in seqs])
    parent = np.zeros(1, np.uint32)
    taxon = np.zeros(len(seqs), np.uint32)
    p = dict(k=16, sketch_size=16, window_len=128, window_stride=113, bucket_cap=3)
    odb = _oracle_db(seq, goffs, p)
    for splits in [None, [5, 6, 12, 22]]:
        db = gpu_build(mc, u8(seq), goffs, parent, taxon, splits=splits, **p)
        _assert_dump_equal(mc, db, odb)
        _assert_stats_equal(db, odb)
        db.free()


def test_live_extension_equals_build_from_scratch(mc):
    """Targets added after a finalize get larger ids; with keep-smallest the
    extended database equals a from-scratch build over all targets."""
    w = synth.mid_workload(seed=11, n_pairs=10, n_families=1, genera_per_family=2, len_scale=0.01, held_genera=0)
    p = dict(w.db_params, bucket_cap=4)
    odb = _oracle_db(w.genomes, w.goffs, p)
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, splits=[3, 9, 15], finalize_each=True, **p)
    _assert_dump_equal(mc, db, odb)
    st, ost = db.stats(), odb.stats()
    for k in ["n_targets", "n_windows", "n_pairs", "n_keys", "n_locations"]:
        assert st[k] == ost[k], k
    db.free()


def test_bucket_cap_keeps_smallest_on_gpu(mc):
    rng = random.Random(9)
    unit = _rand_seq(rng, 113)
    L = 113 * 300 + 15
    seq = (unit * 301)[:L]
    p = dict(k=16, sketch_size=16, window_len=128, window_stride=113, bucket_cap=254)
    seqs = [seq, seq[: 113 * 150 + 15], seq]
    full = "".join(seqs)
    goffs = offsets([len(s) for s in seqs])
    odb = _oracle_db(full, goffs, p)
    db = gpu_build(mc, u8(full), goffs, np.zeros(1, np.uint32), np.zeros(3, np.uint32), **p)
    _assert_dump_equal(mc, db, odb)
    _assert_stats_equal(db, odb)
    assert db.stats()["overflow_keys"] == 16
    db.free()


def test_dump_key_ranges(mc, tiny):
    w = tiny
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    odb = _oracle_db(w.genomes, w.goffs, w.db_params)
    for lo, hi in [(0, 1 << 20), (1 << 28, 1 << 29), (123456789, 123456790), (5, 5)]:
        g = db.dump(lo, hi)
        o = odb.dump(lo, hi)
        for a, b in zip(g, o):
            assert (a == b).all()
    db.free()


def test_default_allocator_path(mc, tiny):
    w = tiny
    mc.use_torch_allocator(False)
    try:
        db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
        odb = _oracle_db(w.genomes, w.goffs, w.db_params)
        _assert_dump_equal(mc, db, odb)
        got = gpu_classify(mc, db, w.reads, w.roffs, w.qoffs, **{k: v for k, v in w.cls_params.items()
                                                                   if k != "max_candidates"})
        want = odb.classify(w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, **w.cls_params)
        for a, b in zip(got[:3], want):
            assert (a == b).all()
        db.free()
    finally:
        mc.use_torch_allocator(True)


# ---------------------------------------------------------------- classify
def _check_classify(mc, db, odb, parent, taxon, reads, roffs, qoffs, m=4, **cp):
    got_l, got_h, got_t, got_c, ctr = gpu_classify(mc, db, reads, roffs, qoffs, with_cands=True, m=m, **cp)
    ol, oh, ot, ost, oc = odb.classify(parent, taxon, reads, roffs, qoffs, max_candidates=m, with_stats=True,
                                       with_cands=True, n_threads=8, **cp)
    assert (got_h == oh).all(), np.nonzero(got_h != oh)[0][:10]
    assert (got_t == ot).all()
    assert (got_c == oc).all()
    assert (got_l == ol).all()
    # counters: features looked up, locations gathered, distinct locations
    assert int(ctr[0]) == int(ost[:, 0].sum())
    assert int(ctr[1]) == int(ost[:, 1].sum())
    assert int(ctr[2]) == int(ost[:, 2].sum())
    return ctr


def test_classify_tiny_matches_oracle(mc, tiny):
    w = tiny
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    odb = _oracle_db(w.genomes, w.goffs, w.db_params)
    cp = {k: v for k, v in w.cls_params.items() if k != "max_candidates"}
    _check_classify(mc, db, odb, w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, **cp)
    db.free()


@pytest.mark.parametrize("m,hits_min,band,max_insert", [(1, 0, 0, 0), (2, 1, 50, 0), (8, 10, 100, 1000),
                                                        (3, 4, 10, 390), (4, 2, 1, 0)])
def test_classify_parameters_match_oracle(mc, m, hits_min, band, max_insert):
    w = synth.mid_workload(seed=21, n_pairs=3000, n_families=1, genera_per_family=2, len_scale=0.02, held_genera=1,
                      held_per_genus=2)
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    odb = _oracle_db(w.genomes, w.goffs, w.db_params)
    _check_classify(mc, db, odb, w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, m=m, hits_min=hits_min,
                    lca_band_pct=band, max_insert=max_insert)
    db.free()


def test_classify_paired_genera_matches_oracle(mc):
    w = synth.mid_workload(seed=1001, n_pairs=20000, n_families=1, genera_per_family=3, len_scale=0.05, held_genera=1,
                      held_per_genus=3)
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    odb = _oracle_db(w.genomes, w.goffs, w.db_params)
    _assert_dump_equal(mc, db, odb)
    cp = {k: v for k, v in w.cls_params.items() if k != "max_candidates"}
    _check_classify(mc, db, odb, w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, **cp)
    db.free()


def test_classify_other_database_parameters(mc):
    w = synth.mid_workload(seed=3, n_pairs=2000, n_families=1, genera_per_family=2, len_scale=0.02, held_genera=0)
    p = dict(k=12, sketch_size=8, window_len=64, window_stride=40, bucket_cap=20)
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **p)
    odb = _oracle_db(w.genomes, w.goffs, p)
    _assert_dump_equal(mc, db, odb)
    _check_classify(mc, db, odb, w.parent, w.taxon_of_target, w.reads, w.roffs, w.qoffs, m=4, hits_min=2,
                    lca_band_pct=20, max_insert=300)
    db.free()


def test_classify_edge_queries(mc, tiny):
    """Empty queries, mates shorter than k, all-N mates, lower case, three
    mates, long reads beyond the shared-memory window budget."""
    w = tiny
    rng = random.Random(8)
    g = bytes(w.genomes).decode()
    mates, qsizes = [], []

    def add(*ms):
        mates.extend(ms)
        qsizes.append(len(ms))

    add()  # no mates
    add("")  # empty mate
    add("ACGTACGTAC")  # shorter than k
    add("N" * 120)
    add(g[1000:1100].lower())
    add(g[5000:5100], g[5200:5300], g[5400:5500])  # three mates
    add(g[300000:301500])  # 1500 bp: 14 windows, large path
    add(g[700000:700150], "")
    for _ in range(50):
        a = rng.randrange(len(g) - 400)
        add(g[a:a + rng.randint(0, 400)], g[a + 50:a + 50 + rng.randint(0, 200)])
    reads = "".join(mates)
    roffs = offsets([len(x) for x in mates])
    qoffs = np.zeros(len(qsizes) + 1, np.uint32)
    qoffs[1:] = np.cumsum(qsizes)
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    odb = _oracle_db(w.genomes, w.goffs, w.db_params)
    ctr = _check_classify(mc, db, odb, w.parent, w.taxon_of_target, reads, roffs, qoffs, m=4, hits_min=4,
                          lca_band_pct=10, max_insert=0)
    assert ctr[3] >= 1  # the 1500 bp read went through the large path
    db.free()


def test_medium_and_large_histogram_paths(mc):
    """300 identical targets: every feature keeps 254 locations, so a 300 bp
    read (three windows) has about 760 distinct locations, beyond the main
    shared-memory histogram (medium path), and a 900 bp read (eight windows)
    about 2,000, beyond the medium one (large path); both must give the
    same answers."""
    rng = random.Random(12)
    base = _rand_seq(rng, 3000)
    n_t = 300
    genomes = base * n_t
    goffs = offsets([len(base)] * n_t)
    parent = np.array([0] + [0] * n_t, np.uint32)
    taxon = np.arange(1, n_t + 1, dtype=np.uint32)
    p = dict(k=16, sketch_size=16, window_len=128, window_stride=113, bucket_cap=254)
    db = gpu_build(mc, u8(genomes), goffs, parent, taxon, **p)
    odb = _oracle_db(genomes, goffs, p)
    reads = [base[a:a + 300] for a in range(0, 2600, 37)] + [base[a:a + 900] for a in range(0, 2000, 97)]
    roffs = offsets([len(r) for r in reads])
    qoffs = np.arange(len(reads) + 1, dtype=np.uint32)
    ctr = _check_classify(mc, db, odb, parent, taxon, "".join(reads), roffs, qoffs, m=8, hits_min=1,
                          lca_band_pct=10, max_insert=0)
    assert ctr[3] > 0 and ctr[6] > 0
    db.free()


def test_wide_location_database_matches_oracle(mc):
    """Target and window ids that do not fit 32 bits together (2^17 + 1
    short targets and one target of 66,372 windows): the database stores
    64-bit locations instead of 32-bit ones, and the dump, the counters and
    the classification must still equal the oracle's."""
    big, big_o = synth.iid_genomes(17, [7_500_000])
    n_small = (1 << 17) + 1
    small, small_o = synth.iid_genomes(18, [24] * n_small, stream_base=0xD000000000)
    genomes = np.concatenate([small, big])
    goffs = np.concatenate([small_o, small_o[-1] + big_o[1:]]).astype(np.uint64)
    n_t = n_small + 1
    # taxonomy: root -> 64 genera -> targets
    parent = np.concatenate([[0], np.zeros(64, np.uint32), 1 + np.arange(n_t) % 64]).astype(np.uint32)
    taxon = np.arange(65, 65 + n_t, dtype=np.uint32)
    p = dict(k=16, sketch_size=16, window_len=128, window_stride=113, bucket_cap=254)
    db = gpu_build(mc, genomes, goffs, parent, taxon, **p)
    odb = _oracle_db(genomes, goffs, p)
    try:
        assert db.stats()["loc_bytes"] == 8
        _assert_dump_equal(mc, db, odb)
        _assert_stats_equal(db, odb)
        reads, roffs, qoffs, _ = synth.simulate_reads(19, 3000, big, big_o, paired=True, len_lo=150, len_hi=150,
                                                      sub=0.01, frag_b=300.0, frag_sd_abs=30.0)
        _check_classify(mc, db, odb, parent, taxon, reads, roffs, qoffs, m=4, hits_min=4, lca_band_pct=10,
                        max_insert=390)
    finally:
        db.free()


def test_query_beyond_window_limit_reports_capacity(mc, tiny):
    w = tiny
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    g = bytes(w.genomes).decode()
    mates = [g[0:100], g[0:113 * 70]]  # the second query has 70 windows
    roffs = offsets([len(x) for x in mates])
    qoffs = np.arange(3, dtype=np.uint32)
    import torch
    label = torch.zeros(2, dtype=torch.int32, device="cuda")
    hits = torch.zeros(2, dtype=torch.int32, device="cuda")
    db.classify(dev(u8("".join(mates))), dev(roffs), dev(qoffs), label=label, hits=hits, **w.cls_params)
    with pytest.raises(mc.McError) as e:
        mc.mc_classify_status(db.handle)
    assert e.value.code == mc.MC_ERR_CAPACITY
    assert host_u32(label)[1] == mc.MC_NO_TAXON
    assert host_u32(label)[0] == w.taxon_of_target[0]
    mc.mc_classify_status(db.handle)  # cleared
    db.free()


def test_classify_before_finalize_is_a_state_error(mc):
    db = mc.Database.create(np.zeros(1, np.uint32))
    import torch
    z = torch.zeros(2, dtype=torch.int64, device="cuda")
    q = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(mc.McError) as e:
        db.classify(torch.zeros(1, dtype=torch.uint8, device="cuda"), z, q)
    assert e.value.code == mc.MC_ERR_STATE
    db.free()


def test_batch_invariance(mc, tiny):
    """A query's answer does not depend on the batch it is classified in."""
    w = tiny
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    cp = {k: v for k, v in w.cls_params.items() if k != "max_candidates"}
    full = gpu_classify(mc, db, w.reads, w.roffs, w.qoffs, **cp)
    for a, b in [(0, 1), (17, 500), (9000, 11000)]:
        lo, hi = int(w.roffs[w.qoffs[a]]), int(w.roffs[w.qoffs[b]])
        ro = w.roffs[w.qoffs[a]:w.qoffs[b] + 1] - np.uint64(lo)
        qo = (w.qoffs[a:b + 1] - w.qoffs[a]).astype(np.uint32)
        part = gpu_classify(mc, db, w.reads[lo:hi], ro, qo, **cp)
        for x, y in zip(full[:3], part[:3]):
            assert (x[a:b] == y).all()
    db.free()


def test_query_mate_and_insert_limits(mc, tiny):
    """More than MC_MAX_QUERY_MATES mates leave the query unclassified with a
    capacity status; max_insert beyond MC_MAX_INSERT is rejected."""
    import torch
    w = tiny
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    g = bytes(w.genomes).decode()
    mates = [g[0:100]] + [g[1000 + 40 * i: 1030 + 40 * i] for i in range(40)]
    roffs = offsets([len(x) for x in mates])
    qoffs = np.array([0, 1, 41], dtype=np.uint32)
    label = torch.zeros(2, dtype=torch.int32, device="cuda")
    hits = torch.zeros(2, dtype=torch.int32, device="cuda")
    db.classify(dev(u8("".join(mates))), dev(roffs), dev(qoffs), label=label, hits=hits, **w.cls_params)
    with pytest.raises(mc.McError) as e:
        mc.mc_classify_status(db.handle)
    assert e.value.code == mc.MC_ERR_CAPACITY
    assert host_u32(label)[1] == mc.MC_NO_TAXON and host_u32(label)[0] == w.taxon_of_target[0]
    with pytest.raises(mc.McError) as e:
        db.classify(dev(u8("".join(mates))), dev(roffs), dev(qoffs), **dict(w.cls_params, max_insert=70000))
    assert e.value.code == mc.MC_ERR_ARG
    db.free()
