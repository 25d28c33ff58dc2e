"""The N > 1 path of bench.py on CPU: two gloo ranks.

On several GPUs the bench runs independent replicas (weak scaling): each rank
solves its own seeded fields, with no collective on the data path; the
process group only synchronises the timed region and takes the slowest
rank's time.  These tests check that host logic with world size 2 on CPU.
"""

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_info()
        dist.barrier()
        # each rank's timed region differs; all must report the slowest one
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, w)
        seeds = bench.rank_seeds(r, 4)
        out.put((r, lr, w, ms, bench.whole_job_value(w, 4, 3, ms), seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_seeds():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, l0, w0, ms0, v0, s0), (r1, l1, w1, ms1, v1, s1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    # max over ranks: both report the slower rank's 15 ms
    assert ms0 == ms1 == 15.0
    # whole-job value: 2 ranks x 4 fields x 3 steps over 15 ms
    assert v0 == v1 == pytest.approx(2 * 4 * 3 / 0.015)
    # replicas solve disjoint fields
    assert not set(s0) & set(s1) and len(set(s0)) == 4


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.whole_job_value(1, 64, 10, 50.0) == pytest.approx(64 * 10 / 0.05)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the reference arm (the CPU oracle) runs and prints on
    rank 0 alone; the other ranks exit without work."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    args = bench.parse()
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args) is None
    assert buf.getvalue() == ""
