"""The benchmark's multi-process logic on CPU ranks (gloo, world size 2 or 3): the
reported time is the maximum over ranks and the work is the sum, and rank
identity comes from the launcher's environment. Each GPU runs an independent
replica of the workload (no collective on the data path), so these are the
only cross-rank operations.
"""
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
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_info()
        t, u = bench.aggregate(10.0 + 5.0 * rank, 1000.0 * (rank + 1), ws)
        out[rank] = (ws, r, local, t, u)
    finally:
        dist.destroy_process_group()


def test_aggregate_max_time_sum_units_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        ws, r, local, t, u = out[rank]
        assert (ws, r, local) == (world, rank, rank)
        assert t == 15.0  # slowest rank
        assert u == 3000.0  # all ranks' atom-steps


def test_single_rank_aggregate_is_identity():
    import bench
    assert bench.aggregate(12.5, 7.0, 1) == (12.5, 7.0)


def test_partition_balances_and_covers():
    import numpy as np
    from paper_1607_02904_gb300 import shard
    rng = np.random.Generator(np.random.Philox(7))
    sizes = rng.integers(64, 4097, size=256)
    for world in (1, 2, 3, 8):
        parts = shard.partition(shard.system_cost(sizes), world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(sizes.size))
        loads = [shard.system_cost(sizes[p]).sum() for p in parts]
        # LPT bound: max load <= mean + largest item
        assert max(loads) <= sum(loads) / world + shard.system_cost(sizes.max())


def _grad_worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_1607_02904_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = torch.arange(8, dtype=torch.float64) * (rank + 1)
        loss = torch.tensor([10.0 * (rank + 1)], dtype=torch.float64)
        shard.allreduce_sum(g, loss)
        out[rank] = (g.tolist(), loss.item())
    finally:
        dist.destroy_process_group()


def test_gradient_allreduce_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_grad_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        g, loss = out[rank]
        assert g == [3.0 * k for k in range(8)]
        assert loss == 30.0


# One data-parallel fitting step over a batch of independent cells: each rank
# evaluates its cost-balanced share of the cells (here with the oracle as the
# evaluation: energies and their complex-step parameter derivatives) and the
# loss and table gradient are summed over ranks. Every rank must end with the
# loss and gradient of the whole batch computed in one process.
FIT_BATCH = dict(n_cells=5, nmin=40, nmax=90, seed_k=11)


def _oracle_loss_grad(cells):
    import numpy as np
    import oracle
    from tests import _systems as S
    table = S.table_for(["Si", "C"], oracle.mix_tersoff89)
    target = table * (1.0 + 0.01 * np.sin(np.arange(table.size)))  # a perturbed table
    loss = torch.zeros(1, dtype=torch.float64)
    grad = torch.zeros(table.size, dtype=torch.float64)
    for x, t, box in cells:
        nl = oracle.neighbors(x, box, 3.0)
        e, _, _ = oracle.compute(x, t, box, table, nl)
        e0, _, _ = oracle.compute(x, t, box, target, nl)
        loss += (e - e0) ** 2
        for p in range(table.size):
            if p % 14 == 0:
                continue
            de, _ = oracle.cs_param(x, t, box, table, nl, p)
            grad[p] += 2.0 * (e - e0) * de
    return loss, grad


def _fit_worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import workloads as W
    from paper_1607_02904_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes, _ = W.batched_cell_sizes(FIT_BATCH["n_cells"], FIT_BATCH["nmin"],
                                        FIT_BATCH["nmax"], FIT_BATCH["seed_k"])
        mine = shard.shard_cells(sizes, world, rank)
        cells = W.batched_cells(**FIT_BATCH, subset=mine)
        loss, grad = shard.fit_step(lambda: _oracle_loss_grad(cells))
        out[rank] = (list(mine), loss.item(), grad.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_fit_step_equals_whole_batch(world):
    import numpy as np
    import workloads as W
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_fit_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    loss_ref, grad_ref = _oracle_loss_grad(W.batched_cells(**FIT_BATCH))
    parts = [out[r][0] for r in range(world)]
    assert sorted(i for p in parts for i in p) == list(range(FIT_BATCH["n_cells"]))
    assert all(len(p) > 0 for p in parts)
    for r in range(world):
        _, loss, grad = out[r]
        assert abs(loss - loss_ref.item()) <= 1e-12 * abs(loss_ref.item())
        g = np.asarray(grad)
        assert np.abs(g - grad_ref.numpy()).max() <= 1e-12 * np.abs(grad_ref.numpy()).max()
