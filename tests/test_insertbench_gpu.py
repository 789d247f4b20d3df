"""The hash-table insert build that bench.py times beside the library's
sort-based build (membench/insertbench.cu, the build primitive of Sections
5.1 and 5.3).  On the window sketches of a small workload it must find as
many distinct features and keep as many locations as the library's
database, and every feature whose locations fit the cap must hold exactly
the windows whose sketch contains it (arrival order, compared sorted)."""
import numpy as np
import pytest

import synth
from gpu_helpers import dev, host_u32

pytestmark = pytest.mark.gpu


def test_hash_insert_build_matches_the_sketches_and_the_database():
    import torch
    import membench
    from paper_2106_08150_gb300 import mc
    mc.use_torch_allocator()
    w = synth.mid_workload(seed=77, n_pairs=10, n_families=1, genera_per_family=3, len_scale=0.05, held_genera=0)
    p = dict(w.db_params, bucket_cap=6)
    db = mc.Database.create(w.parent, **p)
    try:
        db.add_targets(dev(w.genomes), dev(w.goffs), w.taxon_of_target)
        db.finalize()
        st = db.stats()
    finally:
        db.free()
    prm = mc.db_params(**p)
    n_t = w.n_targets
    d_go = dev(w.goffs)
    win = torch.zeros(n_t + 1, dtype=torch.int64, device="cuda")
    mc.mc_window_offsets(prm, n_t, d_go, win)
    torch.cuda.synchronize()
    n_win = int(win[-1].item())
    s = p["sketch_size"]
    sk = torch.empty(n_win * s, dtype=torch.int32, device="cuda")
    cnt = torch.empty(n_win, dtype=torch.int32, device="cuda")
    mc.mc_sketch(prm, n_t, dev(w.genomes), d_go, win, n_win, sk, cnt)
    torch.cuda.synchronize()
    log_slots = int(2 * st["n_keys"]).bit_length()
    r = membench.hash_insert_build(sk, cnt, n_win, s, p["bucket_cap"], log_slots, return_tables=True)
    assert r["n_keys"] == st["n_keys"]
    assert r["n_kept"] == st["n_locations"]

    # expected buckets: windows whose sketch holds the feature, ascending
    sk_h = host_u32(sk).reshape(n_win, s)
    c_h = host_u32(cnt).astype(np.int64)
    valid = np.arange(s)[None, :] < c_h[:, None]
    f_all = sk_h[valid]
    w_all = np.repeat(np.arange(n_win), c_h)
    order = np.lexsort((w_all, f_all))
    f_all, w_all = f_all[order], w_all[order]
    uf, first = np.unique(f_all, return_index=True)
    bounds = np.append(first, len(f_all))
    want = {int(f): w_all[a:b] for f, a, b in zip(uf, bounds[:-1], bounds[1:])}

    t = r["tables"]
    keys = host_u32(t["keys"])
    count = host_u32(t["count"]).astype(np.int64)
    off = t["offset"].cpu().numpy()
    vals = host_u32(t["vals"]).astype(np.int64)
    used = np.nonzero(keys != 0xFFFFFFFF)[0]
    assert sorted(int(keys[i]) for i in used) == sorted(want)
    checked = 0
    for slot in used:
        f, c = int(keys[slot]), int(count[slot])
        assert c == len(want[f])
        kept = vals[off[slot]:off[slot] + min(c, p["bucket_cap"])]
        if c <= p["bucket_cap"]:
            assert (np.sort(kept) == want[f]).all()
            checked += 1
        else:
            assert np.isin(kept, want[f]).all() and len(np.unique(kept)) == len(kept)
    assert checked > 100 and (count > p["bucket_cap"]).any()
