"""The device memory provider contract of mc_set_allocator: blocks must be
256-byte aligned (the kernels use 16- and 32-byte vector accesses from the
start of a block).  A provider that hands out a misaligned block gets it
back through its free callback, and the call fails with MC_ERR_OOM instead
of running kernels on it."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_misaligned_provider_blocks_are_returned_and_rejected():
    import torch
    from paper_2106_08150_gb300 import mc

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    live = {}
    freed = []

    def _alloc(ctx, size, stream):
        base = torch.cuda.caching_allocator_alloc(int(size) + 256, torch.cuda.current_device(), stream or 0)
        p = base + 16  # 16-byte aligned, not 256-byte aligned
        live[p] = base
        return p

    def _free(ctx, ptr, size, stream):
        freed.append(ptr)
        torch.cuda.caching_allocator_delete(live.pop(ptr))

    a = mc.mc_allocator(mc.ALLOC_FN(_alloc), mc.FREE_FN(_free), None)
    mc._check(mc._lib.mc_set_allocator(ctypes.byref(a)))
    try:
        import synth
        w = synth.tiny_workload(n_reads=10, n_decoys=0)
        with pytest.raises(mc.McError) as e:
            db = mc.Database.create(w.parent, **w.db_params)
            db.free()
        assert e.value.code == mc.MC_ERR_OOM
        assert freed and not live  # every block went back to the provider
    finally:
        mc.use_torch_allocator(False)
    torch.cuda.synchronize()
