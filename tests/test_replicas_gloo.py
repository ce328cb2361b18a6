"""The multi-GPU form is replicas only: each rank runs its own simulation and
the bench combines the ranks' work over the slowest rank's time.  This runs the
bench's combining code on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    ws, r, local = bench.dist_setup()
    ms = 10.0 if rank == 0 else 12.5          # the slower rank sets the time
    moves = 1000.0 * (rank + 1)
    bench.barrier(ws)
    ms_max, value, cells = bench.job_rates(ms, moves, 50, 4, ws)
    out[rank] = (ws, r, ms_max, value, cells)
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_as_replicas():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        ws, r, ms_max, value, cells = res[rank]
        assert ws == 2 and r == rank
        assert ms_max == pytest.approx(12.5)
        assert value == pytest.approx(3000.0 / 12.5e-3)      # all ranks' moves over the slowest time
        assert cells == pytest.approx(2 * 50 * 4 / 12.5e-3)
