"""mc_db_finalize failing part-way (Section 4.1 build phase): a refused
allocation before the sort leaves the added targets pending, so the call
can be repeated and gives the same database as an undisturbed build; a
failure after the sort keeps the previously published layout serving
classification and refuses further growth with MC_ERR_STATE.

The allocation failures come from a device memory provider that refuses one
chosen allocation (host side; no kernel is disturbed).  The sort's bounded
wait is made to run out by a test export that makes the last radix pass
skip its first tile, whose counts the next tile then waits for in vain: the
wait gives up after its limit, the kernel records the timeout in a status
word and returns, and the host reports MC_ERR_TIMEOUT (no fault, no hang)."""
import ctypes

import numpy as np
import pytest

import synth
from gpu_helpers import dev, gpu_build, gpu_classify

pytestmark = pytest.mark.gpu


class RefusingProvider:
    """PyTorch-backed provider; `refuse(index, size)` picks one allocation
    (counted from 1 after `arm`) to refuse."""

    def __init__(self, mc):
        import torch
        self.n = 0
        self.refuse = None
        self.refused = 0

        def _alloc(ctx, size, stream):
            self.n += 1
            if self.refuse is not None and self.refuse(self.n, int(size)):
                self.refuse = None
                self.refused += 1
                return None
            return torch.cuda.caching_allocator_alloc(int(size), torch.cuda.current_device(), stream or 0)

        def _free(ctx, ptr, size, stream):
            torch.cuda.caching_allocator_delete(ptr)

        self.a = mc.mc_allocator(mc.ALLOC_FN(_alloc), mc.FREE_FN(_free), None)
        mc._check(mc._lib.mc_set_allocator(ctypes.byref(self.a)))

    def arm(self, refuse):
        self.n = 0
        self.refuse = refuse


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2106_08150_gb300 import mc
    w = synth.tiny_workload(n_reads=2000, n_decoys=200)
    prov = RefusingProvider(mc)
    yield mc, w, prov
    mc.use_torch_allocator(False)


def _add(mc, db, w, a, b):
    lo, hi = int(w.goffs[a]), int(w.goffs[b])
    first = db.add_targets(dev(w.genomes[lo:hi]), dev((w.goffs[a:b + 1] - np.uint64(lo)).astype(np.uint64)),
                           w.taxon_of_target[a:b])
    assert first == a


def _classify(mc, db, w):
    cp = {k: v for k, v in w.cls_params.items() if k != "max_candidates"}
    return gpu_classify(mc, db, w.reads, w.roffs, w.qoffs, m=w.cls_params.get("max_candidates", 4), **cp)[:3]


@pytest.mark.parametrize("which", ["pair buffer", "sort scratch"])
def test_refused_allocation_before_the_sort_can_be_retried(env, which):
    mc, w, prov = env
    ref = gpu_build(mc, w.genomes, w.goffs, w.parent, w.taxon_of_target, **w.db_params)
    want = _classify(mc, ref, w)
    ref.free()

    db = mc.Database.create(w.parent, **w.db_params)
    try:
        _add(mc, db, w, 0, len(w.goffs) - 1)
        # finalize allocates the second pair buffer first, then the sort's scratch
        prov.arm((lambda i, size: i == 1) if which == "pair buffer" else (lambda i, size: i == 2))
        with pytest.raises(mc.McError) as e:
            db.finalize()
        assert e.value.code == mc.MC_ERR_OOM and prov.refused
        prov.arm(None)
        db.finalize()
        for x, y in zip(_classify(mc, db, w), want):
            assert (x == y).all()
    finally:
        db.free()


def test_failure_after_the_sort_keeps_the_published_layout(env):
    mc, w, prov = env
    n = len(w.goffs) - 1
    half = n // 2
    ref = gpu_build(mc, w.genomes[: int(w.goffs[half])], w.goffs[: half + 1], w.parent, w.taxon_of_target[:half],
                    **w.db_params)
    want = _classify(mc, ref, w)
    ref.free()

    db = mc.Database.create(w.parent, **w.db_params)
    try:
        _add(mc, db, w, 0, half)
        db.finalize()
        _add(mc, db, w, half, n)
        # the layout step's first allocation (its 32-byte counters) comes after the sort
        prov.arm(lambda i, size: size == 32)
        with pytest.raises(mc.McError) as e:
            db.finalize()
        assert e.value.code == mc.MC_ERR_OOM and prov.refused
        prov.arm(None)
        with pytest.raises(mc.McError) as e:
            db.finalize()
        assert e.value.code == mc.MC_ERR_STATE
        with pytest.raises(mc.McError) as e:
            _add(mc, db, w, 0, 1)
        assert e.value.code == mc.MC_ERR_STATE
        for x, y in zip(_classify(mc, db, w), want):
            assert (x == y).all()
    finally:
        db.free()


def test_sort_wait_that_runs_out_keeps_the_published_layout(env):
    mc, w, prov = env
    prov.arm(None)
    n = len(w.goffs) - 1
    half = n // 2
    ref = gpu_build(mc, w.genomes[: int(w.goffs[half])], w.goffs[: half + 1], w.parent, w.taxon_of_target[:half],
                    **w.db_params)
    want = _classify(mc, ref, w)
    ref.free()

    with pytest.raises(mc.McError) as e:
        mc.mc_debug_stall_next_sort(10)  # below the allowed range
    assert e.value.code == mc.MC_ERR_ARG
    db = mc.Database.create(w.parent, **w.db_params)
    try:
        _add(mc, db, w, 0, half)
        db.finalize()
        _add(mc, db, w, half, n)
        mc.mc_debug_stall_next_sort(50_000_000)  # 50 ms
        with pytest.raises(mc.McError) as e:
            db.finalize()
        assert e.value.code == mc.MC_ERR_TIMEOUT
        with pytest.raises(mc.McError) as e:
            db.finalize()
        assert e.value.code == mc.MC_ERR_STATE
        with pytest.raises(mc.McError) as e:
            _add(mc, db, w, 0, 1)
        assert e.value.code == mc.MC_ERR_STATE
        for x, y in zip(_classify(mc, db, w), want):
            assert (x == y).all()
    finally:
        db.free()
    # the stall is one-shot: the next build is undisturbed
    again = gpu_build(mc, w.genomes[: int(w.goffs[half])], w.goffs[: half + 1], w.parent, w.taxon_of_target[:half],
                      **w.db_params)
    try:
        for x, y in zip(_classify(mc, again, w), want):
            assert (x == y).all()
    finally:
        again.free()
