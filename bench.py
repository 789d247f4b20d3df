#!/usr/bin/env python3
"""Benchmark of the GB300 MetaCache-GPU hot path.

One step = the whole hot path over one batch of synthetic input: build the
database from the reference genomes (sketch, sort, cap, condensed layout)
and classify every read pair against it (the paper's on-the-fly mode,
Section 6.3).  The default workload is the large single-GPU database:
10,000 genomes (about 14.3 Gbp: 980 genera of bacterial-like genomes plus 200
repeat-rich eukaryote-like genomes that overfill buckets) and 50M
paired-end 2x150 bp reads.  `--workload mid` is the 1,000-genome / 10M-pair
configuration.

Prints one JSON line.  `value` is read pairs classified per second over the
whole step (build included); `build_gbps` and `classify_mreads_s` split it.
The batched mixed-length section and the served section (an offered-load
sweep of the request loop against the plain one-job-per-launch path) run
against the same database.  `--impl reference` times the CPU oracle (the
reference arm of this build) on a bounded sample of the same workload, in
the same unit.

Multi-GPU: the path shards by reads with a replicated database (no data-path
collective), so N ranks run independent replicas (weak scaling).
"""
from __future__ import annotations

import argparse
import math
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "build Gbp/s; classify Mreads/s; served p50/p99 latency, oracle-exact labels"
UNIT = "Mreads/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["large", "mid", "large_small", "small", "tiny"], default="large",
                    help="large = 10,000 genomes (~14.3 Gbp, repeat-rich) / 50M pairs (the measured configuration); "
                         "mid = 1,000 genomes / 10M pairs; large_small (the large recipe at 1/10: ~1.4 Gbp, 2M "
                         "pairs), small and tiny for profiling")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-genera", type=int, default=2)
    ap.add_argument("--cpu-sample-pairs", type=int, default=20000)
    ap.add_argument("--batches", type=int, default=256,
                    help="mixed-length query batches of the batched-classification section (0 = skip)")
    ap.add_argument("--serve-seconds", type=float, default=8.0,
                    help="seconds of arrivals at each offered load of the served section (0 = skip)")
    ap.add_argument("--serve-loads", type=str, default="0.5,0.7,0.9,1.1,1.3",
                    help="offered loads of the served section, as fractions of the tuned batched throughput")
    ap.add_argument("--serve-pool", type=int, default=32, help="distinct jobs the served section cycles through")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shape for the classify kernels")
    ap.add_argument("--no-insert-comparison", action="store_true",
                    help="skip timing the hash-table insert build beside the sort build")
    return ap.parse_args()


# ----------------------------------------------------------------- workload
def make_workload(name: str, rank: int):
    import synth
    if name == "large":
        w = synth.large_workload(seed=1002, scaled=True, held_genera=5, held_per_genus=10)
    elif name == "large_small":
        w = synth.large_workload(seed=1002, scaled=True, n_families=10, n_euk=20, n_pairs=2_000_000, held_genera=1,
                                 held_per_genus=10)
    elif name == "mid":
        w = synth.mid_workload(seed=1001)
    elif name == "small":
        w = synth.mid_workload(seed=1001, n_families=1, genera_per_family=10, n_pairs=1_000_000)
    else:
        w = synth.mid_workload(seed=1001, n_families=1, genera_per_family=2, len_scale=0.1, n_pairs=50_000)
    if rank:
        # replicas classify their own reads against the same database
        reads, roffs, qoffs, truth = synth.simulate_reads(
            1001 + 7919 * rank, w.n_queries, w.genomes, w.goffs, paired=True, len_lo=150, len_hi=150, sub=0.005,
            indel=0.0005, frag_b=300.0, frag_sd_abs=30.0)
        w.reads, w.roffs, w.qoffs, w.truth = reads, roffs, qoffs, truth
    return w


def workload_config(w, args, n_gpus):
    return {
        "workload": w.name,
        "genomes": w.n_targets,
        "genome_bp": w.n_bp,
        "read_pairs": w.n_queries,
        "mate_len": 150,
        "k": w.db_params["k"], "sketch_size": w.db_params["sketch_size"], "window_len": w.db_params["window_len"],
        "window_stride": w.db_params["window_stride"], "bucket_cap": w.db_params["bucket_cap"],
        "max_candidates": w.cls_params["max_candidates"], "hits_min": w.cls_params["hits_min"],
        "lca_band_pct": w.cls_params["lca_band_pct"], "max_insert": w.cls_params["max_insert"],
        "step": "build database from all genomes + classify all read pairs (on-the-fly)",
        "parallelism": f"replicas{n_gpus}" if n_gpus > 1 else "single",
        "l2": (f"inputs larger than L2 (genomes {w.n_bp / 1e9:.1f} GB, reads {w.reads.size / 1e9:.1f} GB)"
               if w.n_bp > (1 << 30) else "small workload"),
        "recipe": w.recipe,
    }


# ------------------------------------------------------------- ranks
def max_over_ranks(vals, world: int, device=None) -> list:
    """Element-wise maximum over all ranks (the timed region's slowest rank)."""
    if world <= 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def whole_job_rate(units_per_rank: float, world: int, steps: int, total_ms: float, scale: float = 1e6) -> float:
    """Units processed by all ranks per second (weak scaling: every rank does
    the same per-rank work), in units of `scale`."""
    return world * units_per_rank * steps / (total_ms * 1e-3) / scale


# ------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ------------------------------------------------------ roofline models
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    return 6800.0, "fallback 6.8 TB/s"


# sources that make up each kernel (a capture's traffic figure is valid
# while these files are unchanged)
_CLASSIFY_SRC = ["mc_classify.cu", "mc_sketch.cuh", "mc_common.cuh"]
_BUILD_SRC = ["mc_build.cu", "mc_sketch.cuh", "mc_common.cuh"]


def kernel_source_hash(kernel: str) -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2106_08150_gb300", "csrc")
    for f in (_CLASSIFY_SRC if kernel.startswith("classify") else _BUILD_SRC):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


# scoring kernels and their block of mc_classify_debug's per-kernel counters
SCORE_KERNELS = {"classify_score": 0, "classify_sort256": 1, "classify_sort512": 2, "classify_sort1024": 3,
                 "classify_sort2048": 6, "classify_medium": 4, "classify_large": 5}


def algorithmic_bytes(kernel: str, w, st: dict, ctr) -> float | None:
    """Algorithmic HBM bytes of ALL launches of `kernel` in one step: every
    input the kernel needs read once and every output written once, random
    probes and bucket reads counted in whole 32-byte sectors."""
    n_win = st["n_windows"]
    s = w.db_params["sketch_size"]
    slots = n_win * s  # emitted pair slots (sentinels included)
    n_real = st["n_pairs"]
    if kernel == "sketch_emit":
        return w.n_bp * 1.0 + slots * 8.0  # read each base once, write the pair slots
    if kernel == "radix_pass":
        return (slots + 3 * n_real) * 8.0 + 4 * n_real * 8.0  # read every input once, write every real pair
    if kernel == "radix_totals":
        return slots * 8.0  # one read of the first pass's input
    if kernel == "fin_count":
        return n_real * 8.0
    if kernel == "fin_emit":
        return n_real * 8.0 + st["n_locations"] * 8.0 + st["n_keys"] * 20.0
    if kernel == "tab_emit":
        return st["n_keys"] * 20.0 + st["n_keys"] * 16.0
    if ctr is None:
        return None
    reads_in = int(w.roffs[-1]) + 8 * (w.n_seq + 1) + 4 * (w.n_queries + 1)
    if kernel == "classify_lookup":
        # bases + offsets, one 32 B table sector per feature, bucket list + metadata out
        return reads_in + 32.0 * float(ctr[0]) + 8.0 * float(ctr[4]) + 16.0 * w.n_queries
    if kernel in SCORE_KERNELS:
        # the queries this kernel finished: metadata + bucket list in, the 32 B
        # sectors of every gathered bucket, 12 B of outputs
        k = SCORE_KERNELS[kernel]
        q, found, sect = (float(ctr[7 + 3 * k + i]) for i in range(3))
        return (16.0 + 12.0) * q + 8.0 * found + 32.0 * sect
    return None


def build_random_roofline(n_bp: int, n_pairs: int, n_locations: int, read32_gbs: float, copy_gbs: float,
                          achieved_gbps: float) -> dict:
    """The build against the HBM random-access roofline, with the method's
    insert model: per pair a 32-byte key-slot update and a 32-byte value
    write at random positions, served at the measured random 32-byte read
    rate; the bases read once and every stored location read and written
    once (16 bytes), streamed at the copy peak."""
    rand_b = 64.0 * n_pairs / n_bp
    stream_b = 1.0 + 16.0 * n_locations / n_bp
    roof = 1.0 / (rand_b / (read32_gbs * 1e9) + stream_b / (copy_gbs * 1e9)) / 1e9
    return {"achieved_gbps": round(achieved_gbps, 2), "roofline_gbps": round(roof, 1),
            "frac": round(achieved_gbps / roof, 4), "random_bytes_per_bp": round(rand_b, 3),
            "stream_bytes_per_bp": round(stream_b, 3), "unit": "Gbp/s"}


def build_rooflines(n_bp: int, st: dict, read32_gbs: float, copy_gbs: float, achieved_gbps: float) -> dict:
    """The build against both rooflines: the sector model (every algorithmic
    byte at the copy peak: 1 B per base read once, per pair a 32-byte
    key-slot update and a 32-byte value write, per stored location 16 B read
    and written once) and the random-access model (the pair bytes at the
    measured random 32-byte read rate, the rest at the copy peak)."""
    sector_b = 1.0 + 64.0 * st["n_pairs"] / n_bp + 16.0 * st["n_locations"] / n_bp
    sector_roof = copy_gbs / sector_b
    return {
        "sector_model": {"bytes_per_bp": round(sector_b, 3), "roofline_gbps": round(sector_roof, 1),
                         "frac": round(achieved_gbps / sector_roof, 4), "peak_gbs": copy_gbs},
        "random_access_model": build_random_roofline(n_bp, st["n_pairs"], st["n_locations"], read32_gbs, copy_gbs,
                                                     achieved_gbps),
        "achieved_gbps": round(achieved_gbps, 2), "unit": "Gbp/s",
    }


def load_traffic():
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return {}
    try:
        return json.load(open(p))
    except ValueError:
        return {}


# ----------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_2106_08150_gb300 import mc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    mc.use_torch_allocator()
    t_gen = time.time()
    w = make_workload(args.workload, rank)
    t_gen = time.time() - t_gen
    stream = torch.cuda.Stream(device=dev)

    def to_dev(a):
        a = np.ascontiguousarray(a)
        if a.dtype == np.uint64:
            a = a.view(np.int64)
        elif a.dtype == np.uint32:
            a = a.view(np.int32)
        return torch.from_numpy(a).to(dev)

    g, go = to_dev(w.genomes), to_dev(w.goffs)
    r, ro, qo = to_dev(w.reads), to_dev(w.roffs), to_dev(w.qoffs)
    nq = w.n_queries
    label = torch.empty(nq, dtype=torch.int32, device=dev)
    hits = torch.empty(nq, dtype=torch.int32, device=dev)
    top = torch.empty(nq, dtype=torch.int32, device=dev)
    cp = mc.classify_params(**w.cls_params)
    torch.cuda.synchronize()

    tuned = None

    def step(seq_g, off_g, seq_r, off_r, off_q, evs=None):
        db = mc.Database.create(w.parent, stream=stream, **w.db_params)
        if tuned is not None:
            mc.mc_db_set_tuning(db.handle, tuned)
        db.add_targets(seq_g, off_g, w.taxon_of_target)
        db.finalize()
        if evs is not None:
            evs.append(torch.cuda.Event(enable_timing=True))
            evs[-1].record(stream)
        mc.mc_classify(db.handle, cp, w.n_seq, seq_r, off_r, nq, off_q, label, hits, top, stream=stream)
        db.free()  # synchronises the database stream
        return db

    # untimed: database statistics, the launch shape of the classify kernels
    # (the autotuner on the first 2^20 pairs; any shape gives the same
    # labels) and the classify counters of that shape, for the roofline
    db = mc.Database.create(w.parent, stream=stream, **w.db_params)
    db.add_targets(g, go, w.taxon_of_target)
    db.finalize()
    st = db.stats()
    n_s = min(nq, 1 << 20)
    sample = [mc.batch(int(w.qoffs[n_s]), r, ro, qo[: n_s + 1], label, hits, top)]
    if not args.no_autotune:
        tuned, tune_rec = mc.mc_autotune(db.handle, cp, sample, reps=2)
        mc.mc_db_set_tuning(db.handle, tuned)
    ctr = torch.zeros(mc.MC_DEBUG_COUNTERS, dtype=torch.int64, device=dev)
    mc.mc_classify_debug(db.handle, cp, w.n_seq, r, ro, nq, qo, label, hits, top, None, ctr, stream=stream)
    mc.mc_classify_status(db.handle, stream)
    ctr = ctr.cpu().numpy()
    db.free()
    torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(g, go, r, ro, qo)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    clocks.start()
    mc.mc_trace_report(reset=True)
    mc.mc_trace_enable(True)
    launches0 = mc.mc_kernel_launches()
    ev_start = torch.cuda.Event(enable_timing=True)
    ev_end = torch.cuda.Event(enable_timing=True)
    mids, starts = [], []
    ev_start.record(stream)
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        starts.append(e0)
        step(g, go, r, ro, qo, mids)
    ev_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches = mc.mc_kernel_launches() - launches0
    mc.mc_trace_enable(False)
    trace = mc.mc_trace_report(reset=True)
    clk = clocks.stop()
    total_ms = ev_start.elapsed_time(ev_end)
    build_ms = sum(a.elapsed_time(b) for a, b in zip(starts, mids))
    ends = starts[1:] + [ev_end]
    cls_ms = sum(a.elapsed_time(b) for a, b in zip(mids, ends))

    total_ms, build_ms, cls_ms = max_over_ranks([total_ms, build_ms, cls_ms], world, dev)

    # end-to-end through the public API with host buffers (pinned), copies
    # timed every step.  The genome copy is split into chunks on a copy
    # stream so that adding chunk i overlaps copying chunk i+1; the reads
    # follow in parts, each classified (its own mc_classify call into its
    # slice of the outputs) as soon as it has arrived.
    e2e = None
    if not args.no_e2e:
        n_chunks = 8
        cut = np.searchsorted(w.goffs, np.linspace(0, w.n_bp, n_chunks + 1)).clip(0, w.n_targets)
        cut[0], cut[-1] = 0, w.n_targets
        cut = np.unique(cut)
        chunks = [(int(a), int(b)) for a, b in zip(cut[:-1], cut[1:]) if b > a]
        hg = torch.from_numpy(w.genomes).pin_memory()
        hgo = [torch.from_numpy((w.goffs[a:b + 1] - w.goffs[a]).view(np.int64)).pin_memory() for a, b in chunks]
        hr = torch.from_numpy(w.reads).pin_memory()
        rparts = [(qa, qb, nm, ba, bb, torch.from_numpy(ro.view(np.int64)).pin_memory(),
                   torch.from_numpy(qo.view(np.int32)).pin_memory())
                  for qa, qb, nm, ba, bb, ro, qo in read_parts(w.roffs, w.qoffs, 4)]
        hl = torch.empty(nq, dtype=torch.int32).pin_memory()
        hh = torch.empty(nq, dtype=torch.int32).pin_memory()
        dg = torch.empty_like(hg, device=dev)
        dgo = [torch.empty_like(x, device=dev) for x in hgo]
        dr = torch.empty_like(hr, device=dev)
        dparts = [(torch.empty_like(ho, device=dev), torch.empty_like(hq, device=dev)) for *_, ho, hq in rparts]
        h2d = sum(x.numel() * x.element_size() for x in [hg, hr] + hgo + [t for *_, ho, hq in rparts for t in (ho, hq)])
        d2h = 2 * nq * 4
        copy_stream = torch.cuda.Stream(device=dev)

        phases = []

        def e2e_step():
            evs = []
            with torch.cuda.stream(copy_stream):
                for (a, b), ho, do in zip(chunks, hgo, dgo):
                    lo, hi = int(w.goffs[a]), int(w.goffs[b])
                    dg[lo:hi].copy_(hg[lo:hi], non_blocking=True)
                    do.copy_(ho, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(copy_stream)
                    evs.append(ev)
                ev_parts = []
                for (qa, qb, nm, ba, bb, ho, hq), (do_, dq_) in zip(rparts, dparts):
                    dr[ba:bb].copy_(hr[ba:bb], non_blocking=True)
                    do_.copy_(ho, non_blocking=True)
                    dq_.copy_(hq, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(copy_stream)
                    ev_parts.append(ev)
            tp = [time.perf_counter()]
            db = mc.Database.create(w.parent, stream=stream, **w.db_params)
            if tuned is not None:
                mc.mc_db_set_tuning(db.handle, tuned)
            for (a, b), do, ev in zip(chunks, dgo, evs):
                stream.wait_event(ev)
                lo = int(w.goffs[a])
                db.add_targets(dg[lo:], do, w.taxon_of_target[a:b])
            tp.append(time.perf_counter())
            db.finalize()
            tp.append(time.perf_counter())
            for (qa, qb, nm, ba, bb, ho, hq), (do_, dq_), ev in zip(rparts, dparts, ev_parts):
                stream.wait_event(ev)
                mc.mc_classify(db.handle, cp, nm, dr[ba:], do_, qb - qa, dq_, label[qa:qb], hits[qa:qb], top[qa:qb],
                               stream=stream)
            with torch.cuda.stream(stream):
                hl.copy_(label, non_blocking=True)
                hh.copy_(hits, non_blocking=True)
            db.free()
            stream.synchronize()
            tp.append(time.perf_counter())
            phases.append([round((b_ - a_) * 1e3, 1) for a_, b_ in zip(tp[:-1], tp[1:])])

        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        step_ms = []
        for _ in range(args.steps):
            t1 = time.perf_counter()
            e2e_step()
            step_ms.append(round((time.perf_counter() - t1) * 1e3, 1))
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks([(time.perf_counter() - t0) * 1e3], world, dev)[0]
        # the host-to-device copy alone (genomes + reads, one stream)
        t1 = time.perf_counter()
        with torch.cuda.stream(copy_stream):
            dg.copy_(hg, non_blocking=True)
            dr.copy_(hr, non_blocking=True)
        copy_stream.synchronize()
        h2d_gbs = (hg.numel() + hr.numel()) / (time.perf_counter() - t1) / 1e9
        e2e = {"value": whole_job_rate(nq, world, args.steps, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": e2e_ms / args.steps, "step_ms": step_ms, "h2d_alone_gbs": round(h2d_gbs, 1),
               "phase_ms_add_finalize_classify": phases[-args.steps:]}

    # roofline of the dominant kernel
    kernels = {k: {"launches": n, "total_ms": ms, "avg_ms": ms / max(n, 1)} for k, (n, ms) in trace.items()}
    dom = max(kernels, key=lambda k: kernels[k]["total_ms"]) if kernels else None
    peak, peak_src = measured_peaks()
    roof = None
    if dom:
        per_step_bytes = algorithmic_bytes(dom, w, st, ctr)
        per_launch_count = kernels[dom]["launches"] / args.steps
        traffic_db = load_traffic()
        traffic = None
        tinfo = traffic_db.get(dom)
        if per_step_bytes is not None:
            per_launch_bytes = per_step_bytes / per_launch_count
            if tinfo and tinfo.get("src_sha") == kernel_source_hash(dom):
                # DRAM bytes of one ncu capture (profiles/), scaled to this
                # launch by the ratio of algorithmic bytes; null once the
                # kernel sources changed after the capture
                ratio = tinfo["dram_bytes_per_launch_captured"] / tinfo["algorithmic_bytes_per_launch_captured"]
                traffic = round(ratio * per_launch_bytes)
            achieved = per_launch_bytes / (kernels[dom]["avg_ms"] * 1e-3) / 1e9
            roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(achieved / peak, 4), "traffic": traffic,
                    "algorithmic_bytes_per_launch": per_launch_bytes, "peak_source": peak_src + " (burst)"}

    # random-access roofline: the feature-table probes and bucket gathers
    # read 16-32 bytes at random positions, which HBM serves far below the
    # copy bandwidth; measured here on this GPU (8 GiB buffer, 2^28 reads)
    import membench
    rand = {w_: round(membench.random_read_gbs(8 << 30, w_, 1 << 28, stream.cuda_stream), 1) for w_ in (16, 32)}
    rand_roof = {"read16_gbs": rand[16], "read32_gbs": rand[32], "unit": "GB/s",
                 "note": "best of 6 shapes of random aligned reads of 16 / 32 bytes, 8 GiB buffer; the classify "
                         "kernels' algorithmic bytes count 32-byte sectors, so they are compared with read32_gbs"}
    for kname in ["classify_lookup", *SCORE_KERNELS]:
        if kname in kernels:
            b = algorithmic_bytes(kname, w, st, ctr)
            per = kernels[kname]["launches"] / args.steps
            if b is not None and per:
                ach = b / per / (kernels[kname]["avg_ms"] * 1e-3) / 1e9
                rand_roof[kname] = {"achieved_gbs": round(ach, 1), "frac_of_read32": round(ach / rand[32], 4)}
    build_ach = world * w.n_bp * args.steps / (build_ms * 1e-3) / 1e9
    rand_roof["build"] = build_random_roofline(w.n_bp, st["n_pairs"], st["n_locations"], rand[32], peak, build_ach)

    value = whole_job_rate(nq, world, args.steps, total_ms)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(w, args, world),
        "build_gbps": round(build_ach, 3),
        "classify_mreads_s": round(world * nq * args.steps / (cls_ms * 1e-3) / 1e6, 3),
        "classify_mates_mreads_s": round(world * w.n_seq * args.steps / (cls_ms * 1e-3) / 1e6, 3),
        "build_ms_per_step": round(build_ms / args.steps, 3), "classify_ms_per_step": round(cls_ms / args.steps, 3),
        "db": {k: st[k] for k in ["n_targets", "n_windows", "n_pairs", "n_keys", "n_locations", "overflow_keys",
                                  "dropped_locations", "table_slots", "max_probe", "load_factor", "device_bytes"]},
        "build_roofline": build_rooflines(w.n_bp, st, rand[32], peak, build_ach),
        "classify_counters": {"features": int(ctr[0]), "locations": int(ctr[1]), "distinct_locations": int(ctr[2]),
                              "large_path_queries": int(ctr[3]), "medium_path_queries": int(ctr[6]),
                              "features_found": int(ctr[4]),
                              "bucket_sectors": int(ctr[5]),
                              "per_kernel": {k: {"queries": int(ctr[7 + 3 * i]), "found": int(ctr[8 + 3 * i]),
                                                 "sectors": int(ctr[9 + 3 * i])}
                                             for k, i in SCORE_KERNELS.items() if int(ctr[7 + 3 * i])}},
        "roofline": roof,
        "random_access_roofline": rand_roof,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "kernels": {k: {"launches": v["launches"], "avg_ms": round(v["avg_ms"], 4),
                        "share": round(v["total_ms"] / max(sum(x["total_ms"] for x in kernels.values()), 1e-9), 4)}
                    for k, v in kernels.items()},
        "clocks": clk,
        "generation_s": round(t_gen, 1),
        "classify_tuning": tuned.as_dict() if tuned is not None else "default",
    }
    if w.held is not None and world == 1:
        out["extension"] = run_extension(w, dev, stream, tuned)
    if world == 1 and not args.no_insert_comparison:
        out["build_insert_comparison"] = run_insert_comparison(w, dev, stream, kernels, args.steps, st)
    if args.batches and world == 1:
        out["batched"] = run_batched(args, w, dev, stream)
    if args.serve_seconds > 0 and world == 1 and w.held is not None:
        rate = out.get("batched", {}).get("graph_tuned", {}).get("mreads_s")
        out["served"] = run_served_sweep(args, w, dev, stream, rate, tuned)
    return out, w


def read_parts(roffs: np.ndarray, qoffs: np.ndarray, n_parts: int) -> list:
    """The queries split into n_parts consecutive parts for classification
    in pieces: per part (q_a, q_b, mates, b_a, b_b, roffs, qoffs) with its
    queries [q_a, q_b), its bases [b_a, b_b) of the read array and its mate
    and query offsets rebased to start at 0 (u64 / u32), so that each part is
    one self-contained mc_classify call on reads[b_a:]."""
    nq = len(qoffs) - 1
    qcut = np.linspace(0, nq, n_parts + 1).astype(np.int64)
    out = []
    for qa, qb in zip(qcut[:-1], qcut[1:]):
        ma, mb = int(qoffs[qa]), int(qoffs[qb])
        ba, bb = int(roffs[ma]), int(roffs[mb])
        ro = (roffs[ma:mb + 1] - np.uint64(ba)).astype(np.uint64)
        qo = (qoffs[qa:qb + 1] - np.uint32(ma)).astype(np.uint32)
        out.append((int(qa), int(qb), mb - ma, ba, bb, ro, qo))
    return out


# ------------------------------------------- build primitive comparison
# kernels of the library's build after sketching: sort (digit totals and
# four radix passes) and layout (finalize and feature table)
SORT_BUILD_KERNELS = {"sort": ["radix_totals", "radix_pass"],
                      "layout": ["fin_count", "fin_emit", "tab_dispmax", "exclusive_max_i64", "tab_emit",
                                 "scan_tile_sums", "scan_downsweep"]}


def run_insert_comparison(w, dev, stream, kernels, steps, st, reps: int = 2):
    """The paper's build primitive (a hash table keyed by feature, filled
    with warp-aggregated atomics, Sections 5.1 and 5.3) against the
    library's sort-based build, on the same pairs: the sketches of all the
    workload's windows.  The hash build is membench.hash_insert_build
    (count, scan, fill; last of `reps` runs); the sort build's times are
    its kernels in the timed step (CUDA events).  Both exclude sketching."""
    import torch
    import membench
    from paper_2106_08150_gb300 import mc
    p = w.db_params
    prm = mc.db_params(**p)
    n_t = w.n_targets
    d_g = torch.from_numpy(w.genomes).to(dev)
    d_go = torch.from_numpy(w.goffs.view(np.int64)).to(dev)
    win = torch.zeros(n_t + 1, dtype=torch.int64, device=dev)
    mc.mc_window_offsets(prm, n_t, d_go, win, stream=stream)
    stream.synchronize()
    n_win = int(win[-1].item())
    s = p["sketch_size"]
    sk = torch.empty(max(1, n_win * s), dtype=torch.int32, device=dev)
    cnt = torch.empty(max(1, n_win), dtype=torch.int32, device=dev)
    mc.mc_sketch(prm, n_t, d_g, d_go, win, n_win, sk, cnt, stream=stream)
    stream.synchronize()
    del d_g
    log_slots = int(st["table_slots"]).bit_length() - 1
    res = None
    for _ in range(reps):
        res = membench.hash_insert_build(sk, cnt, n_win, s, p["bucket_cap"], log_slots, stream=stream)
        torch.cuda.empty_cache()
    sort = {}
    for part, names in SORT_BUILD_KERNELS.items():
        sort[part + "_ms"] = round(sum(kernels[k]["total_ms"] for k in names if k in kernels) / steps, 3)
    sort["total_ms"] = round(sort["sort_ms"] + sort["layout_ms"], 3)
    return {"pairs": int(st["n_pairs"]), "hash_insert": res, "sort_build": sort,
            "same_keys": res["n_keys"] == int(st["n_keys"]), "same_kept": res["n_kept"] == int(st["n_locations"]),
            "note": "hash insert: count (atomicCAS/atomicAdd, warp-aggregated by __match_any_sync) + exclusive scan "
                    "+ fill (atomic cursors), buckets in arrival order, cap keeps the first arrivals; sort build: "
                    "radix sort + finalize + feature table, buckets ordered, cap keeps the smallest; sketching "
                    "excluded from both"}


# ------------------------------------------------------ live extension
def run_extension(w, dev, stream, tuned, reps: int = 3):
    """Live extension of the resident database (Section 4.1: new targets get
    the next ids): the held-out genomes (new species of existing genera) are
    added to a finalized database of all the workload's genomes and the
    database is finalized again; the new pairs are sorted and merged into
    the stored ones.  Wall time of each call (both leave the database
    stream idle), median of `reps` fresh databases; the build from scratch
    of the same genomes is timed beside it."""
    import torch
    from paper_2106_08150_gb300 import mc
    hblob, hoffs, htaxon = w.held
    d_h, d_ho = torch.from_numpy(hblob).to(dev), torch.from_numpy(hoffs.view(np.int64)).to(dev)
    d_g, d_go = torch.from_numpy(w.genomes).to(dev), torch.from_numpy(w.goffs.view(np.int64)).to(dev)
    rec = []
    for _ in range(reps):
        db = mc.Database.create(w.parent, stream=stream, **w.db_params)
        t0 = time.perf_counter()
        db.add_targets(d_g, d_go, w.taxon_of_target)
        db.finalize()
        t1 = time.perf_counter()
        p0 = db.stats()["n_pairs"]
        t2 = time.perf_counter()
        db.add_targets(d_h, d_ho, htaxon)
        t3 = time.perf_counter()
        db.finalize()
        t4 = time.perf_counter()
        st = db.stats()
        db.free()
        rec.append((t1 - t0, t3 - t2, t4 - t3, st["n_pairs"] - p0, p0))
    med = lambda i: float(np.median([r[i] for r in rec]))
    return {"added_genomes": len(htaxon), "added_bp": int(hoffs[-1]), "added_pairs": int(rec[-1][3]),
            "stored_pairs": int(rec[-1][4]), "add_ms": round(med(1) * 1e3, 2), "finalize_ms": round(med(2) * 1e3, 2),
            "extension_ms": round((med(1) + med(2)) * 1e3, 2), "build_from_scratch_ms": round(med(0) * 1e3, 2),
            "reps": reps,
            "note": "finalize sorts only the new pairs and merges them into the stored ones (no re-sort); the "
                    "layout is rewritten in one streaming pass"}


# ------------------------------------------------------ batched queries
def run_batched(args, w, dev, stream):
    """Mixed-length query batches against the resident database: one
    mc_classify call per batch, one launch set over all batches
    (mc_classify_batches), a CUDA-graph plan, and the plan with the
    autotuner's launch shape.  All four must give identical outputs."""
    import torch
    import synth
    from paper_2106_08150_gb300 import mc

    t0 = time.time()
    batches = synth.mixed_batches(1003, w.genomes, w.goffs, n_batches=args.batches)
    gen_s = time.time() - t0
    db = mc.Database.create(w.parent, stream=stream, **w.db_params)
    db.add_targets(torch.from_numpy(w.genomes).to(dev), torch.from_numpy(w.goffs.view(np.int64)).to(dev),
                   w.taxon_of_target)
    db.finalize()
    cp = mc.classify_params(**dict(w.cls_params, max_insert=0))

    def t(a):
        a = np.ascontiguousarray(a)
        a = a.view(np.int64) if a.dtype == np.uint64 else a.view(np.int32) if a.dtype == np.uint32 else a
        return torch.from_numpy(a).to(dev)

    ins, ref, out = [], [], []
    for reads, roffs, qoffs, _ in batches:
        nq = len(qoffs) - 1
        ins.append((len(roffs) - 1, nq, t(reads) if len(reads) else torch.zeros(1, dtype=torch.uint8, device=dev),
                    t(roffs), t(qoffs)))
        ref.append([torch.empty(max(1, nq), dtype=torch.int32, device=dev) for _ in range(3)])
        out.append([torch.empty(max(1, nq), dtype=torch.int32, device=dev) for _ in range(3)])
    descs = [mc.batch(n_seq, seq, offs, qo, *o) for (n_seq, nq, seq, offs, qo), o in zip(ins, out)]
    total_q = sum(x[1] for x in ins)
    total_mates = sum(x[0] for x in ins)
    total_bp = sum(int(b[1][-1]) for b in batches)
    torch.cuda.synchronize()

    def per_batch(outs):
        for (n_seq, nq, seq, offs, qo), o in zip(ins, outs):
            if nq:
                mc.mc_classify(db.handle, cp, n_seq, seq, offs, nq, qo, *o, stream=stream)

    # each variant: warm-up runs, then timed runs (fewer than the main step's
    # counts, so that the section stays short on the large database)
    n_warm, n_time = max(1, min(args.warmup, 2)), max(1, min(args.steps, 5))

    def timed(fn):
        for _ in range(n_warm):
            fn()
        torch.cuda.synchronize()
        n0 = mc.mc_kernel_launches()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n_time):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / n_time
        return {"mreads_s": round(total_q / (ms * 1e-3) / 1e6, 3), "ms": round(ms, 3),
                "launches": (mc.mc_kernel_launches() - n0) // n_time, "runs": n_time}

    def same():
        mc.mc_classify_status(db.handle, stream)
        return all(bool(torch.equal(x[:n], y[:n])) for (_, n, *_r), rx, ox in zip(ins, ref, out)
                   for x, y in zip(rx, ox))

    # untimed: counters of all batches and a per-kernel trace of one launch set
    ctr = torch.zeros(mc.MC_DEBUG_COUNTERS, dtype=torch.int64, device=dev)
    for (n_seq, nq, seq, offs, qo), o in zip(ins, out):
        if nq:
            mc.mc_classify_debug(db.handle, cp, n_seq, seq, offs, nq, qo, *o, None, ctr, stream=stream)
    mc.mc_classify_status(db.handle, stream)
    ctr = [int(x) for x in ctr.cpu()]
    mc.mc_trace_report(reset=True)
    mc.mc_trace_enable(True)
    mc.mc_classify_batches(db.handle, cp, descs, stream=stream)
    torch.cuda.synchronize()
    mc.mc_trace_enable(False)
    trace = {k: round(ms, 3) for k, (n, ms) in mc.mc_trace_report(reset=True).items()}

    res = {}
    res["per_batch"] = timed(lambda: per_batch(ref))
    res["one_launch_set"] = timed(lambda: mc.mc_classify_batches(db.handle, cp, descs, stream=stream))
    ok = same()
    plan = mc.Plan(db.handle, cp, len(descs), total_q)
    res["graph"] = timed(lambda: plan.run(descs, stream))
    ok = ok and same()
    plan.free()
    # autotune on the leading batches (up to 2^20 queries)
    sample, n = [], 0
    for d, x in zip(descs, ins):
        if n + x[1] > (1 << 20):
            break
        sample.append(d)
        n += x[1]
    t0 = time.time()
    best, rec = mc.mc_autotune(db.handle, cp, sample, reps=3)
    tune_s = time.time() - t0
    plan = mc.Plan(db.handle, cp, len(descs), total_q, best)
    res["graph_tuned"] = timed(lambda: plan.run(descs, stream))
    ok = ok and same()
    plan.free()
    db.free()
    sizes = [x[1] for x in ins]
    return {
        "workload": f"{len(batches)} batches, sizes lognormal(median 5e4, sigma 1) in [1e3, 2e6], read length "
                    f"U(50,300), half single-end half pairs, against the {w.name} database",
        "batches": len(batches), "queries": total_q, "mates": total_mates, "bases": total_bp,
        "batch_size_min": int(min(sizes)), "batch_size_max": int(max(sizes)),
        "unit": "Mreads/s", **res, "identical_results": bool(ok), "tuning": best.as_dict(),
        "counters": {"features": ctr[0], "locations": ctr[1], "distinct_locations": ctr[2],
                     "large_path_queries": ctr[3], "medium_path_queries": ctr[6], "features_found": ctr[4],
                     "bucket_sectors": ctr[5]},
        "kernel_ms_one_launch_set": trace,
        "autotune_s": round(tune_s, 2), "autotune_sample_queries": n,
        "autotune_times_ms": [[r[0], r[1], round(r[2], 4)] for r in rec],
        "generation_s": round(gen_s, 1),
    }


# ------------------------------------------------------------ served loop
def run_served_sweep(args, w, dev, stream, batched_rate_mreads_s: float | None, tuned):
    """Request loop over the resident database (mc_server) at several
    offered loads (fractions of the tuned batched throughput): Poisson job
    arrivals, job sizes lognormal (median 1e5, sigma 1.5) in [1e3, 5e6], read
    lengths U(75, 250), half single-end half pairs, 5% of reads from
    not-yet-inserted species; the held-out species are inserted live in two
    extensions during each run.  The same arrival sequence is then replayed
    in full through the plain path (one mc_classify call per job, copies in
    and out, one job at a time)."""
    import torch
    import synth
    from paper_2106_08150_gb300 import mc

    rng = np.random.default_rng(1004)
    t0 = time.time()
    sizes = np.clip(np.round(np.exp(rng.normal(math.log(1e5), 1.5, args.serve_pool))), 1e3, 5e6).astype(np.int64)
    pool = synth.mixed_batches(1004, w.genomes, w.goffs, sizes=sizes, len_lo=75, len_hi=250, held=w.held,
                               held_frac=0.05)
    gen_s = time.time() - t0
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    jobs = [(len(r[1]) - 1, len(r[2]) - 1, pin(r[0]), pin(r[1].view(np.int64)), pin(r[2].view(np.int32)))
            for r in pool]
    max_q = max(j[1] for j in jobs)
    mean_q = float(np.mean(sizes))
    ring = 64
    outs = [[torch.empty(max_q, dtype=torch.int32).pin_memory() for _ in range(3)] for _ in range(ring)]
    hblob, hoffs, htaxon = w.held
    n_held = len(htaxon)
    ext_cut = [0, n_held // 2, n_held]
    cp = mc.classify_params(**dict(w.cls_params, max_insert=0))
    base_rate = batched_rate_mreads_s or 50.0
    d_g, d_go = torch.from_numpy(w.genomes).to(dev), torch.from_numpy(w.goffs.view(np.int64)).to(dev)
    d_out = [torch.empty(max_q, dtype=torch.int32, device=dev) for _ in range(3)]
    dur = args.serve_seconds

    def fresh_db():
        db = mc.Database.create(w.parent, stream=stream, **w.db_params)
        if tuned is not None:
            mc.mc_db_set_tuning(db.handle, tuned)
        db.add_targets(d_g, d_go, w.taxon_of_target)
        db.finalize()
        return db

    def extend(srv, i):
        a, b = ext_cut[i], ext_cut[i + 1]
        lo, hi = int(hoffs[a]), int(hoffs[b])
        srv.extend(hblob[lo:hi], hoffs[a:b + 1] - np.uint64(lo), htaxon[a:b])

    def one_load(frac, seed):
        r = np.random.default_rng(seed)
        rate_q = frac * base_rate * 1e6
        rate_jobs = rate_q / mean_q
        n_arr = max(1, int(r.poisson(rate_jobs * dur)))
        arrivals = np.sort(r.uniform(0, dur, n_arr))
        which = r.integers(0, len(jobs), n_arr)
        ext_at = [dur / 3, 2 * dur / 3]
        db = fresh_db()
        srv = mc.Server(db.handle, cp, n_streams=3)
        n0 = mc.mc_kernel_launches()
        ids, next_ext = [], 0
        t_start = time.perf_counter()
        for k, (ta, jb) in enumerate(zip(arrivals, which)):
            while next_ext < 2 and time.perf_counter() - t_start >= ext_at[next_ext]:
                extend(srv, next_ext)
                next_ext += 1
            delay = ta - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            if k >= ring:
                srv.wait(ids[k - ring])  # the output slot is free again
            n_seq, nq, seq, offs, qo = jobs[jb]
            o = outs[k % ring]
            ids.append(srv.submit(n_seq, seq, offs, qo, o[0], o[1], o[2]))
        while next_ext < 2:
            extend(srv, next_ext)
            next_ext += 1
        srv.drain()
        wall = time.perf_counter() - t_start
        st = srv.stats()
        launches = mc.mc_kernel_launches() - n0
        # the last jobs ran on the final database: replay them alone and compare
        last = [(k, ids[k]) for k in range(max(0, len(ids) - 3), len(ids))]
        infos = {k: srv.wait(i) for k, i in last}
        srv.free()
        same, checked = True, 0
        for k, info in infos.items():
            if info["epoch"] != 2:
                continue
            n_seq, nq, seq, offs, qo = jobs[which[k]]
            out = [torch.empty(nq, dtype=torch.int32, device=dev) for _ in range(3)]
            mc.mc_classify(db.handle, cp, n_seq, seq.to(dev), offs.to(dev), nq, qo.to(dev), *out, stream=stream)
            stream.synchronize()
            same = same and all(bool(torch.equal(x.cpu(), y[:nq])) for x, y in zip(out, outs[k % ring]))
            checked += 1
        # plain path: the same arrivals on the final database, one job at a time
        lat, q_done = [], 0
        t_start = time.perf_counter()
        for ta, jb in zip(arrivals, which):
            delay = ta - (time.perf_counter() - t_start)
            if delay > 0:
                time.sleep(delay)
            n_seq, nq, seq, offs, qo = jobs[jb]
            with torch.cuda.stream(stream):
                ds, do, dq = (seq.to(dev, non_blocking=True), offs.to(dev, non_blocking=True),
                              qo.to(dev, non_blocking=True))
                mc.mc_classify(db.handle, cp, n_seq, ds, do, nq, dq, *d_out, stream=stream)
                for x, y in zip(outs[0], d_out):
                    x[:nq].copy_(y[:nq], non_blocking=True)
            stream.synchronize()
            lat.append(time.perf_counter() - t_start - ta)
            q_done += nq
        plain_wall = time.perf_counter() - t_start
        db.free()
        lat = np.sort(np.array(lat))
        return {
            "offered_load": frac, "offered_mreads_s": round(rate_q / 1e6, 3), "offered_jobs_s": round(rate_jobs, 2),
            "jobs": int(st["jobs_done"]), "queries": int(st["queries_done"]),
            "served": {"throughput_mreads_s": round(st["queries_done"] / max(st["busy_s"], 1e-9) / 1e6, 3),
                       "extension_mean_ms": round(st["extension_mean_s"] * 1e3, 2),
                       "extension_max_ms": round(st["extension_max_s"] * 1e3, 2),
                       "wall_s": round(wall, 2), "p50_latency_s": round(st["p50_latency_s"], 4),
                       "p99_latency_s": round(st["p99_latency_s"], 4),
                       "max_latency_s": round(st["max_latency_s"], 4), "launch_sets": int(st["launch_sets"]),
                       "gpu_launches": int(launches), "extensions": int(st["extensions"]),
                       "hbm_peak_bytes": int(st["hbm_peak"]), "hbm_limit_bytes": int(st["hbm_limit"])},
            "plain_one_job_per_launch": {
                "throughput_mreads_s": round(q_done / plain_wall / 1e6, 3), "wall_s": round(plain_wall, 2),
                "p50_latency_s": round(float(lat[len(lat) // 2]), 4),
                "p99_latency_s": round(float(lat[min(len(lat) - 1, int(0.99 * (len(lat) - 1) + 0.5))]), 4)},
            "final_epoch_jobs_identical_alone": bool(same), "final_epoch_jobs_checked": checked,
        }

    loads = [float(x) for x in args.serve_loads.split(",") if x.strip()]
    curve = [one_load(f, 1004 + i) for i, f in enumerate(loads)]
    sat_served = max(c["served"]["throughput_mreads_s"] for c in curve)
    sat_plain = max(c["plain_one_job_per_launch"]["throughput_mreads_s"] for c in curve)
    return {
        "workload": f"Poisson job arrivals, job size lognormal(median 1e5, sigma 1.5) in [1e3, 5e6], read length "
                    f"U(75,250), half single-end half pairs, 5% from held-out species; {n_held} held-out species "
                    f"genomes inserted live in 2 extensions per run; database {w.name}",
        "seconds_per_load": dur, "base_rate_mreads_s": round(base_rate, 3),
        "base_rate_source": "batched graph_tuned throughput" if batched_rate_mreads_s else "fixed 50 Mreads/s",
        "curve": curve, "saturation_mreads_s": {"served": sat_served, "plain_one_job_per_launch": sat_plain},
        "pool_jobs": len(jobs), "generation_s": round(gen_s, 1),
    }


# ------------------------------------------------------------ CPU arms
def oracle_sample(w, n_targets: int, n_pairs: int):
    """A bounded slice of the workload: the first n_targets genomes (a genus
    is 10 genomes) and read pairs drawn from them, generated like the full
    reads."""
    import synth
    n_t = min(w.n_targets, n_targets)
    hi = int(w.goffs[n_t])
    genomes, goffs = w.genomes[:hi], w.goffs[:n_t + 1].copy()
    reads, roffs, qoffs, _ = synth.simulate_reads(
        4242, n_pairs, genomes, goffs, paired=True, len_lo=150, len_hi=150, sub=0.005, indel=0.0005, frag_b=300.0,
        frag_sd_abs=30.0)
    return genomes, goffs, reads, roffs, qoffs, n_t


def time_oracle(w, n_targets: int, n_pairs: int, threads: int = 0):
    import oracle
    cores = threads or os.cpu_count() or 1
    genomes, goffs, reads, roffs, qoffs, n_t = oracle_sample(w, n_targets, n_pairs)
    t0 = time.perf_counter()
    odb = oracle.DB(genomes, goffs, n_threads=cores, **w.db_params)
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    odb.classify(w.parent, w.taxon_of_target, reads, roffs, qoffs, n_threads=cores, **w.cls_params)
    tc = time.perf_counter() - t0
    bp = int(goffs[-1])
    # scale each half to the full workload
    t_full = tb * (w.n_bp / bp) + tc * (w.n_queries / n_pairs)
    value = w.n_queries / t_full / 1e6
    sample = (f"oracle build of {n_t} genomes ({bp / 1e6:.1f} Mbp, {tb:.2f} s) + classify of {n_pairs} pairs "
              f"({tc:.2f} s) on {cores} threads, each scaled to the full workload ({w.n_bp / 1e9:.2f} Gbp, "
              f"{w.n_queries} pairs)")
    return {"value": round(value, 5), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "build_gbps": round(bp / tb / 1e9, 5), "classify_mreads_s": round(n_pairs / tc / 1e6, 5)}, tb + tc


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, bounded sample per step."""
    w = make_workload(args.workload, 0)
    n_gen, n_pairs = max(1, args.cpu_sample_genera // 2), max(1000, args.cpu_sample_pairs // 4)
    for _ in range(args.warmup):
        time_oracle(w, 10 * n_gen, n_pairs)
    vals, secs = [], 0.0
    last = None
    for _ in range(args.steps):
        last, s = time_oracle(w, 10 * n_gen, n_pairs)
        vals.append(last["value"])
        secs += s
    value = statistics.median(vals)
    cb = dict(last, value=value)
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(w, args, world), "cpu_baseline": cb,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------------------ main
def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, rank, world)), flush=True)
        return 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out, w = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            cb, _ = time_oracle(w, 10 * args.cpu_sample_genera, args.cpu_sample_pairs)
            one, _ = time_oracle(w, 2, 2000, threads=1)
            cb["single_thread"] = {k: one[k] for k in ("value", "sample", "build_gbps", "classify_mreads_s")}
            out["cpu_baseline"] = cb
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
