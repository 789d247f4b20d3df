"""Databases partitioned by target over several GPUs (Sections 4.2 and 4.3).

The paper splits the reference targets over the GPUs of a node: each GPU
builds a database of its own targets, every query batch goes to every
partition, and the partitions' top candidates are merged into one list per
read.  Here each rank (one process per GPU) holds a contiguous range of
target ids, in rank order.  The bucket cap is that of one database of all
targets: a shard keeps at most cap - prior(f) of its locations of feature
f, prior(f) being f's locations in the earlier shards, which the shards
exchange once after adding their targets (mc_db_feature_counts,
mc_db_finalize_after).  Classification runs on every shard and the per-shard
top-m lists are merged by mc_merge_candidates, so the labels equal those of
the single database.

The exchanges are torch.distributed collectives (NCCL between GPUs, gloo on
CPU); the protocol functions drive any shard object with the four methods of
`GpuShard`, so that the same exchange code can be run on CPU ranks.
"""
from __future__ import annotations

import json

import numpy as np


def shard_ranges(goffs: np.ndarray, world: int) -> list[tuple[int, int]]:
    """Contiguous target ranges [lo, hi) for `world` shards, cut so that the
    shards hold about equal numbers of bases (every shard gets at least one
    target when there are enough)."""
    goffs = np.asarray(goffs, dtype=np.uint64)
    n = len(goffs) - 1
    total = float(goffs[-1])
    cuts = [0]
    for r in range(1, world):
        c = int(np.searchsorted(goffs, np.uint64(total * r / world)))
        if n >= world:  # at least one target for this shard and each later one
            c = min(max(c, cuts[-1] + 1), n - (world - r))
        c = min(max(c, cuts[-1]), n)
        cuts.append(c)
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def all_gather_varlen(t, group=None) -> list:
    """Every rank's 1-D tensor `t` (lengths may differ), in rank order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(x.item()) for x in sizes]
    width = max(max(sizes), 1)
    padded = torch.zeros(width, dtype=t.dtype, device=t.device)
    padded[: t.numel()] = t.reshape(-1)
    out = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(out, padded, group=group)
    return [o[:s] for o, s in zip(out, sizes)]


def build_partitioned(shard, group=None):
    """Finalizes this rank's shard with the single-database bucket cap: the
    feature counts of all shards are gathered and each shard is finalized
    against those of the shards before it."""
    import torch.distributed as dist
    rank = dist.get_rank(group)
    keys, counts = shard.feature_counts()
    all_keys = all_gather_varlen(keys, group)
    all_counts = all_gather_varlen(counts, group)
    shard.finalize_after([(all_keys[r], all_counts[r]) for r in range(rank)])


def classify_partitioned(shard, reads, roffs, qoffs, group=None, **cparams):
    """Classifies the same queries on every shard and merges the top-m lists
    (every rank gets the merged result).  Returns (label, hits, top_target,
    cands[n_q, m, 4]) with global target ids."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    cands = shard.classify_cands(reads, roffs, qoffs, **cparams)
    lists = [torch.empty_like(cands) for _ in range(world)]
    dist.all_gather(lists, cands, group=group)
    base = torch.tensor([shard.merge_base], dtype=torch.int64, device=cands.device)
    bases = [torch.zeros_like(base) for _ in range(world)]
    dist.all_gather(bases, base, group=group)
    return shard.merge(lists, [int(b.item()) for b in bases], **cparams)


class GpuShard:
    """One rank's shard on its GPU: targets [base, base + n) of the global
    target list.  Device tensors in, device tensors out."""

    def __init__(self, mc, parent, base: int, seq, offs, taxon, taxon_global, stream=None, **db_params):
        self.mc = mc
        self.merge_base = int(base)  # global id of local target 0
        self.taxon_global = taxon_global  # device, taxa of all global targets
        self.stream = stream
        self.db = mc.Database.create(parent, stream=stream, **db_params)
        self.db.add_targets(seq, offs, taxon)

    def feature_counts(self):
        import torch
        mc = self.mc
        n = mc.mc_db_feature_counts(self.db.handle)
        dev = self.taxon_global.device
        keys = torch.empty(max(1, n), dtype=torch.int32, device=dev)
        counts = torch.empty(max(1, n), dtype=torch.int32, device=dev)
        mc.mc_db_feature_counts(self.db.handle, keys, counts, n)
        return keys[:n], counts[:n]

    def finalize_after(self, prior):
        self.mc.mc_db_finalize_after(self.db.handle, [(k, c, k.numel()) for k, c in prior])

    def classify_cands(self, seq, offs, qoffs, *, max_candidates, **cparams):
        import torch
        nq = qoffs.numel() - 1
        dev = seq.device
        cands = torch.zeros(max(1, nq) * max_candidates * 4, dtype=torch.int32, device=dev)
        self.db.classify(seq, offs, qoffs, cands=cands, stream=self.stream, max_candidates=max_candidates, **cparams)
        self.mc.mc_classify_status(self.db.handle, self.stream)
        return cands

    def merge(self, lists, bases, *, max_candidates, **cparams):
        import torch
        mc = self.mc
        nq = lists[0].numel() // (4 * max_candidates)
        dev = lists[0].device
        label = torch.empty(max(1, nq), dtype=torch.int32, device=dev)
        hits = torch.empty_like(label)
        top = torch.empty_like(label)
        cands = torch.empty(max(1, nq) * max_candidates * 4, dtype=torch.int32, device=dev)
        cp = mc.classify_params(max_candidates=max_candidates, **cparams)
        mc.mc_merge_candidates(self.db.handle, cp, nq, lists, bases, self.taxon_global, self.taxon_global.numel(),
                               label, hits, top, cands, stream=self.stream)
        return label[:nq], hits[:nq], top[:nq], cands[: nq * max_candidates * 4].reshape(nq, max_candidates, 4)

    def save(self, path: str):
        """Writes this shard (Section 4.3: each GPU keeps its partition): its
        condensed layout at `path` (mc_db_save) and its global id base at
        `path + ".shard.json"`."""
        self.db.save(path)
        with open(path + ".shard.json", "w") as f:
            json.dump({"merge_base": self.merge_base}, f)

    @classmethod
    def load(cls, mc, path: str, taxon_global, stream=None) -> "GpuShard":
        """A shard written by save(), ready to classify and merge (its
        database finalized; taxon_global as in the constructor)."""
        with open(path + ".shard.json") as f:
            meta = json.load(f)
        s = cls.__new__(cls)
        s.mc = mc
        s.merge_base = int(meta["merge_base"])
        s.taxon_global = taxon_global
        s.stream = stream
        s.db = mc.Database.load(path, stream=stream)
        return s

    def free(self):
        self.db.free()
