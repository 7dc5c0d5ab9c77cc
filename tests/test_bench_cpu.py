"""bench.py host logic without a GPU: the max-over-ranks reduction on a
two-rank gloo group, and the reference arm (the CPU oracle) on rank 0 only."""
import json
import os
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    out[rank] = bench.reduce_max(1.5 + rank)
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        assert dict(out) == {0: 2.5, 1: 2.5}


def _run_bench(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, env=env, timeout=600)


def test_reference_arm_prints_one_line_on_rank0_only():
    p = _run_bench({"RANK": "1", "WORLD_SIZE": "2"}, "--impl", "reference", "--steps", "1",
                   "--warmup", "3", "--ref-rows", "2")
    assert p.returncode == 0 and p.stdout.strip() == ""
    p = _run_bench({"RANK": "0", "WORLD_SIZE": "1"}, "--impl", "reference", "--steps", "2",
                   "--warmup", "3", "--ref-rows", "2")
    assert p.returncode == 0, p.stderr
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "Mpix/s" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_sweep_radius_list_parsing():
    from paper_1405_1020_gb300 import sweep
    assert sweep._parse_radii("1-10") == list(range(1, 11))
    assert sweep._parse_radii("2,4,8") == [2, 4, 8]
