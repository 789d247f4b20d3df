"""Host-side logic of bench.py's multi-rank path, on CPU with gloo ranks:
max over ranks, whole-job rate, and the reference arm's rank behaviour."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    vals = bench.max_over_ranks([10.0 * (rank + 1), 5.0 - rank], world)
    out.put((rank, vals))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [20.0, 5.0]


def test_whole_job_rate_is_weak_scaling_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.whole_job_rate(10_000_000, 1, 5, 1000.0)
    two = bench.whole_job_rate(10_000_000, 2, 5, 1000.0)
    assert one == pytest.approx(50.0) and two == pytest.approx(100.0)
    assert bench.max_over_ranks([1, 2], 1) == [1.0, 2.0]


def test_reference_arm_non_zero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                        "--steps", "1", "--warmup", "0", "--cpu-sample-pairs", "2000"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "Mreads/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_build_random_roofline_arithmetic():
    import bench
    # every base a pair (64 random bytes) and a location (16 streamed bytes
    # + the base): 1 / (64 / 100 + 17 / 1000) Gbp/s at 100 and 1000 GB/s
    r = bench.build_random_roofline(10**9, 10**9, 10**9, 100.0, 1000.0, 0.5)
    assert r["random_bytes_per_bp"] == 64.0 and r["stream_bytes_per_bp"] == 17.0
    assert abs(r["roofline_gbps"] - round(1.0 / (0.64 + 0.017), 1)) < 1e-9
    assert abs(r["frac"] - round(0.5 / (1.0 / 0.657), 4)) < 1e-9
    # the mid workload's counts at the measured rates give about 155 Gbp/s
    m = bench.build_random_roofline(3_680_156_920, 521_089_020, 521_089_020, 1517.0, 6801.0, 93.7)
    assert 150.0 < m["roofline_gbps"] < 160.0 and 0.55 < m["frac"] < 0.65


def test_algorithmic_bytes_of_the_sort_kernels():
    import types
    import bench
    w = types.SimpleNamespace(db_params={"sketch_size": 16}, n_bp=1000)
    st = {"n_windows": 10, "n_pairs": 150}
    # 160 pair slots in the first pass, 150 real pairs in the other three
    assert bench.algorithmic_bytes("radix_totals", w, st, None) == 160 * 8
    assert bench.algorithmic_bytes("radix_pass", w, st, None) == (160 + 3 * 150) * 8 + 4 * 150 * 8
