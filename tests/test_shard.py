"""Multi-process path of the batched workload, on CPU: the greedy
partition of independent systems over ranks, and a world-size-2 gloo job in
which each rank solves its share with the oracle and rank 0 gathers the
per-system reports (no collective in the data path, one gather at the
end)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synthetic as S
from paper_2609_40159_gb300 import shard


def test_partition_is_a_balanced_cover():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        costs = rng.integers(1, 10_000, size=257).tolist()
        share = shard.partition(costs, world)
        flat = sorted(m for s in share for m in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[m] for m in s) for s in share]
        assert max(loads) <= sum(costs) / world + max(costs)
        assert share == shard.partition(costs, world)  # deterministic


def test_partition_edge_cases():
    assert shard.partition([], 3) == [[], [], []]
    assert shard.partition([5], 2) == [[0], []]
    assert shard.partition([3, 3, 3, 3], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        shard.partition([1], 0)


def test_gather_without_process_group():
    assert shard.gather_reports({"a": 1}) == [{"a": 1}]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    items = S.batch_spec(nmat=12, seed=41, n_lo=200, n_hi=3000, dtype=np.float64)
    costs = [shard.system_cost(it.A.n, it.A.nnz, it.nrhs) for it in items]
    mine = shard.local_share(costs, rank, world)
    report = {"rank": rank, "systems": {}}
    for m in mine:
        it = items[m]
        x = oracle.solve(it.A, it.b)
        res = np.abs(it.A.dense() @ x - it.b).max()
        report["systems"][m] = {"residual": float(res), "n": it.A.n}
    got = shard.gather_reports(report, dist)
    if rank == 0:
        with open(os.path.join(outdir, "gathered.txt"), "w") as f:
            for r in got:
                for m, v in sorted(r["systems"].items()):
                    f.write(f"{r['rank']} {m} {v['residual']:.3e} {v['n']}\n")
    dist.destroy_process_group()


def test_two_rank_gloo_job(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    lines = (tmp_path / "gathered.txt").read_text().split("\n")
    rows = [ln.split() for ln in lines if ln]
    systems = sorted(int(r[1]) for r in rows)
    assert systems == list(range(12))  # every system solved exactly once
    assert {r[0] for r in rows} == {"0", "1"}  # both ranks did work
    assert max(float(r[2]) for r in rows) < 1e-10
