"""Allocation-free classification (mc_classify_noalloc) against mc_classify.

mc_classify_noalloc serves callers that cannot allocate device memory while
they classify (for example a server whose GPU memory is entirely reserved by
another allocator); it works in a fixed scratch array inside the library.
This file is named to be collected last, so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import synth
from gpu_helpers import dev, gpu_build, offsets, u8

pytestmark = pytest.mark.gpu


def test_noalloc_matches_classify_on_two_calls_in_a_row():
    import torch
    from paper_2106_08150_gb300 import mc

    w = synth.tiny_workload(n_reads=4000, n_decoys=400)
    db = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    try:
        # the tiny read set plus long single-end reads whose 14 windows take
        # the large-histogram path (its scratch lives in the fixed array too)
        reads = bytes(w.reads).decode()
        g = bytes(w.genomes).decode()
        mates = [reads[int(w.roffs[i]):int(w.roffs[i + 1])] for i in range(w.n_seq)]
        mates += [g[a:a + 1500] for a in range(0, 1_500_000, 75_000)]
        roffs = offsets([len(x) for x in mates])
        qoffs = np.arange(len(mates) + 1, dtype=np.uint32)
        nq = len(mates)
        d_r, d_ro, d_qo = dev(u8("".join(mates))), dev(roffs), dev(qoffs)
        cp = mc.classify_params(**w.cls_params)

        ref = [torch.empty(nq, dtype=torch.int32, device="cuda") for _ in range(3)]
        mc.mc_classify(db.handle, cp, nq, d_r, d_ro, nq, d_qo, *ref)
        mc.mc_classify_status(db.handle)
        counters = torch.zeros(mc.MC_DEBUG_COUNTERS, dtype=torch.int64, device="cuda")
        dbg = [torch.empty(nq, dtype=torch.int32, device="cuda") for _ in range(3)]
        mc.mc_classify_debug(db.handle, cp, nq, d_r, d_ro, nq, d_qo, *dbg, None, counters)
        mc.mc_classify_status(db.handle)
        assert int(counters[3]) >= 20  # the long reads used the large path

        for _ in range(2):  # the shared scratch keeps the last call's contents
            out = [torch.full((nq,), -7, dtype=torch.int32, device="cuda") for _ in range(3)]
            mc.mc_classify_noalloc(db.handle, cp, nq, d_r, d_ro, nq, d_qo, *out)
            mc.mc_classify_status(db.handle)
            for a, b in zip(ref, out):
                assert torch.equal(a, b)

        too_many = mc.MC_NOALLOC_MAX_QUERIES + 1
        with pytest.raises(mc.McError) as e:
            mc.mc_classify_noalloc(db.handle, cp, nq, d_r, d_ro, too_many, d_qo, *ref)
        assert e.value.code == mc.MC_ERR_CAPACITY
    finally:
        db.free()
