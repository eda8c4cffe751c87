"""The N>1 bench path on CPU: two gloo ranks (127.0.0.1) run the bench's
rank reductions (max of the step times, sum of the work) and the reference
arm's rank-0-only rule.  The solve itself runs as independent replicas, so
the data path has no collective to test."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, _ = bench.dist_env()
        assert (ws, r) == (world, rank)
        bench.barrier(dist)
        t_max = bench.allreduce_max(dist, 1.5 + rank)          # per-rank step times
        work = bench.allreduce_sum(dist, 10.0 * (rank + 1))    # per-rank DOF*iterations
        # the reference arm: only rank 0 runs and prints; other ranks return at once
        ref = None
        if rank == 1:
            class A:
                steps, warmup, ref_subdomains, gpus = 1, 0, 1, world
            ref = bench.reference_arm(A())
        out[rank] = (t_max, work, ref)
    finally:
        dist.destroy_process_group()


def test_two_rank_reductions_and_rank0_only_reference():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.5                        # max over ranks
    assert res[0][1] == res[1][1] == 30.0                       # whole-job sum
    assert res[1][2] is None
