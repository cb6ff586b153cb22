"""The multi-rank path of the benchmark on CPU (gloo, world size 2): ranks simulate disjoint
realisations and the whole-job throughput is the cell-steps of all ranks over the slowest rank's
time, with no data-path collective."""
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


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [2.0, 3.0][rank]  # the second rank is slower
    value, total = bench.weak_scaling_value(local, 1.2e10, device="cpu")
    out[rank] = (value, total, bench.realisation_offset(rank, 256))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_two_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][1] == res[1][1] == 3.0  # max over ranks
    assert res[0][0] == pytest.approx(2 * 1.2e10 / 3.0)
    assert res[0][0] == res[1][0]
    assert {res[0][2], res[1][2]} == {0, 256}  # disjoint realisation keys


def test_single_rank_value():
    import bench
    value, total = bench.weak_scaling_value(2.0, 1e10)
    assert total == 2.0 and value == pytest.approx(5e9)
