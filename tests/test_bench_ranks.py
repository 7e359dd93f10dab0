"""The benchmark's multi-rank host logic on the CPU: two `gloo` ranks on 127.0.0.1.

Under torch.distributed.run every rank advances its own film replica; the whole-job figures are
the slowest rank's time and the sum of all ranks' evaluations.  The reference arm runs on rank 0
only; the other ranks leave without work.
"""
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


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir, per_rank):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sec, n_rhs, e2e = per_rank[rank]
        out = bench.combine_ranks(dist, sec, n_rhs, e2e, "cpu")
        with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
            json.dump(out, f)
    finally:
        dist.destroy_process_group()


def _run_ranks(tmp_path, per_rank):
    world = len(per_rank)
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path), per_rank))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert codes == [0] * world, codes
    return [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]


def test_two_ranks_take_slowest_time_and_sum_evaluations(tmp_path):
    per_rank = [(1.25, 40, 30.0), (2.5, 37, 28.0)]
    got = _run_ranks(tmp_path, per_rank)
    # every rank ends with the same whole-job figures
    assert got[0] == got[1]
    sec_all, rhs_all, e2e_all = got[0]
    assert sec_all == 2.5
    assert rhs_all == 77.0
    assert e2e_all == 58.0
    # value = all ranks' evaluations over the slowest rank's time
    assert rhs_all / sec_all == pytest.approx(30.8)


def test_single_rank_is_the_identity():
    import bench
    assert bench.combine_ranks(None, 1.5, 12, 7.0, "cpu") == (1.5, 12.0, 7.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "2", "--warmup", "3"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
