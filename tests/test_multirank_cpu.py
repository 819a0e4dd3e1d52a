"""Multi-rank host logic of bench.py on CPU: world size 2 over gloo.

Every rank runs its own realisation (no data-path collective); ranks meet only at the
timing barrier and the max-over-ranks reduction, and rank 0 alone prints.  These tests
run that logic with CPU tensors and the gloo backend, without a GPU."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank step times: rank r is slower on the first value, faster on the second
        mine = [1.0 + rank, 10.0 - rank, 3.5]
        dist.barrier()
        got = bench.max_over_ranks(dist, mine, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(rank))
        rate = bench.whole_job_rate(512 ** 3, world, got[0])
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
            json.dump(dict(got=got, seeds=seeds, rate=rate), fh)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_seeds_world2(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["got"] == [2.0, 10.0, 3.5]                 # the slowest rank's time per entry
        assert r["seeds"] == [1, 2]                        # one distinct realisation per rank
        assert r["rate"] == pytest.approx(2 * 512 ** 3 / 2e-3)   # all ranks' particles / max time


def test_max_over_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, [1, 2.5], "cpu") == [1.0, 2.5]
    assert bench.whole_job_rate(100, 1, 1000.0) == pytest.approx(100.0)


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    """`bench.py --impl reference` under torchrun: rank 0 times the oracle sample and
    prints one JSON line; rank 1 exits 0 without work."""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=str(tmp_path), timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
