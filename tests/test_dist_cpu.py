"""The multi-rank path on CPU (gloo, world size 2): ranks simulate disjoint realisations; the
whole-job throughput is the cell-steps of all ranks over the slowest rank's time; and the loop
observables of the whole ensemble come from two small all-reduces (per-sample sums, then four
jackknife sums), equal to the single-process statistics of all realisations."""
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


def _loop_samples():
    import numpy as np
    rng = np.random.default_rng(11)
    n_half, R = 150, 20
    H = np.concatenate([np.linspace(300, -300, n_half + 1), np.linspace(-300, 300, n_half + 1)[1:]])
    k = np.arange(len(H))
    S = np.stack([np.where(k <= n_half, np.tanh((H + h) / 40.0), np.tanh((H - h) / 40.0))
                  for h in rng.normal(90.0, 10.0, size=R)]).astype(np.float32)
    S += rng.normal(0, 0.03, size=S.shape).astype(np.float32)
    return H, n_half, S


def _stats_worker(rank, world, port, out, split):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1912_00310_gb300 import ensemble
    H, n_half, S = _loop_samples()
    mine = S[:split] if rank == 0 else S[split:]  # uneven split (split 0: rank 0 holds none)
    d = ensemble.loop_stats(mine, H, n_half, mode=1, zeta=0.81935)
    out[rank] = {k: d[k] for k in ("Hc_Oe", "Hc_se_Oe", "area_Oe", "area_se_Oe", "area0_Oe", "n_real")}
    out[f"mean{rank}"] = d["mean"].tolist()
    out[f"se{rank}"] = d["mean_se"].tolist()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("split", [7, 0])
def test_loop_statistics_over_two_ranks(split):
    import numpy as np
    from paper_1912_00310_gb300 import build
    build.build()
    import paper_1912_00310_gb300 as P
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_stats_worker, args=(2, port, out, split), nprocs=2, join=True)
        res = dict(out)
    H, n_half, S = _loop_samples()
    ref = P.loop_stats(S, H, n_half, mode=1, zeta=0.81935)
    for r in (0, 1):
        assert res[r]["n_real"] == S.shape[0]
        for key in ("Hc_Oe", "Hc_se_Oe", "area_Oe", "area_se_Oe", "area0_Oe"):
            assert res[r][key] == pytest.approx(ref[key], rel=1e-10), (r, key)
    S64 = S.astype(np.float64)
    assert np.allclose(res["mean0"], S64.mean(0), rtol=0, atol=1e-12)
    assert np.allclose(res["se1"], S64.std(0, ddof=1) / np.sqrt(S.shape[0]), rtol=1e-9, atol=1e-15)
