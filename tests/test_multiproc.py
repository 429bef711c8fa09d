"""The N > 1 host path of bench.py (replicas only: one independent map and view batch per rank,
no collective in the data path) with world size 2 on the gloo backend, on CPU: the timed region
is the slowest rank's, every rank agrees on it, and the job throughput counts both replicas."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [120.0, 180.5][rank]
    total = bench.max_over_ranks(local_ms, world, "cpu")
    # each replica draws its own scene and views
    sc, _, cams = bench.make_workload(2000, 0, rank)
    out[rank] = (total, bench.job_mpix(world, 1000, 10, total), float(sc.planes()[0, :8].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_count_both_replicas():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
        res = dict(out)
    assert res[0][0] == res[1][0] == pytest.approx(180.5)
    assert res[0][1] == pytest.approx(2 * 1000 * 10 / 0.1805 / 1e6)
    assert res[0][2] != res[1][2]      # independent replicas: different scenes per rank
