"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): the slowest rank's time
decides, the whole-job value sums the ranks' work, and only rank 0 runs the reference arm."""
import contextlib
import io
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank times its own problem; the job's time is the slowest rank's
        t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, device="cpu")
        v = bench.whole_job_gdofs(world, 1000, 3.0, t)
        buf = io.StringIO()

        class A:
            steps, warmup = 1, 0
        if rank != 0:
            with contextlib.redirect_stdout(buf):
                bench.run_reference(A, rank, world)
        out[rank] = (t, v, buf.getvalue())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert set(out.keys()) == {0, 1}
    for r in range(world):
        t, v, printed = out[r]
        assert t == 15.0                              # max over ranks
        assert abs(v - 2 * 1000 * 3.0 / 15.0 / 1e9) < 1e-18
    assert out[1][2] == ""                            # rank 1 runs no reference work, prints nothing
