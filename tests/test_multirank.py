"""Multi-rank logic of bench.py on CPU ranks (gloo, world size 2): the timed
value is the slowest rank's time, the value aggregates all ranks' node
updates, every rank takes its own balanced share of the cases, and the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank)
    spec = bench.workload_spec("hartmann_batch", rank, world)
    units = bench.sum_over_ranks(spec["fluid"])
    keys = [(p["W"], p["Ha"], p["q"]) for p in spec["params"]]
    q.put((rank, ms, units, spec["fluid"], keys, bench.whole_job_mlups(units, 100, ms)))
    dist.destroy_process_group()


def test_ranks_share_the_cases_and_aggregate_with_gloo():
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=300) for _ in procs])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    allp = bench.hartmann_draws(2)
    total = sum(p["W"] * p["W"] for p in allp)
    seen = []
    for rank, ms, units, mine, keys, mlups in out:
        assert ms == 15.0                                        # the slower rank sets the time
        assert units == total                                    # node updates of both ranks
        assert abs(mlups - total * 100 / 15e-3 / 1e6) < 1e-6
        assert 0.95 < mine / (total / 2) < 1.05                  # balanced by node count
        seen += keys
    # every case of the 2 x 64 draws on exactly one rank; batch 0 is the 64-case configuration
    assert sorted(seen) == sorted((p["W"], p["Ha"], p["q"]) for p in allp)
    one = bench.workload_spec("hartmann_batch", 0, 1)
    assert len(one["params"]) == 64 and one["fluid"] == 6842872


def test_partition_is_balanced_and_complete():
    sys.path.insert(0, ROOT)
    import bench
    sizes = [7, 1, 5, 5, 3, 9, 2, 2, 8]
    for world in (1, 2, 3, 4):
        parts = bench.partition(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


@pytest.mark.parametrize("workload", ["hartmann_batch"])
def test_reference_arm_line_on_rank_zero(workload):
    """The reference arm prints one line with the same config as the GPU arm
    and loads no product library (the oracle's only)."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    code = ("import runpy, sys, json; sys.argv = ['bench.py', '--impl', 'reference', '--steps', '2', '--warmup', "
            "'1', '--workload', %r]\n"
            "try:\n    runpy.run_path(%r, run_name='__main__')\nexcept SystemExit:\n    pass\n"
            "maps = open('/proc/self/maps').read()\n"
            "print(json.dumps({'product_loaded': 'liblbm_gb300' in maps}))\n") % (
        workload, os.path.join(ROOT, "bench.py"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    line = json.loads(lines[-2])
    assert json.loads(lines[-1]) == {"product_loaded": False}
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "MLUPS"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    sys.path.insert(0, ROOT)
    import bench
    assert line["config"] == bench.spec_config(bench.workload_spec(workload))
