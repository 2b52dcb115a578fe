"""Sharding of the batched workload over ranks (CPU): the cost-balanced
partition, and a world_size-2 gloo run in which each rank solves its share of
a small batch with the oracle and rank 0 gathers and checks the whole batch
against a serial solve.  No GPU and no collective on the data path."""
import os
import socket

import numpy as np
import pytest

from paper_2008_08825_gb300 import inputs, shard


def test_partition_is_exact_and_deterministic():
    sizes = inputs.batched_sizes()
    for world in (1, 2, 3, 4, 8):
        parts = shard.partition_by_cost(sizes, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        assert parts == shard.partition_by_cost(sizes, world)


def test_partition_balance_bound():
    """Greedy list scheduling: max load <= mean load + largest single cost;
    on the 512-instance workload the spread is far tighter (< 1% at 8 ranks)."""
    sizes = inputs.batched_sizes()
    cost_max = float(np.max(sizes.astype(np.float64) ** 3))
    for world in (2, 4, 8):
        ld = shard.loads(sizes, shard.partition_by_cost(sizes, world))
        mean = sum(ld) / world
        assert max(ld) <= mean + cost_max
        assert max(ld) / mean - 1.0 < 0.01


def test_partition_edge_cases():
    assert shard.partition_by_cost([], 3) == [[], [], []]
    assert shard.partition_by_cost([5, 5], 4) == [[0], [1], [], []]
    # the largest instance goes first, to rank 0; equal costs go to the lowest rank
    assert shard.partition_by_cost([2, 9, 2, 2], 2) == [[1], [0, 2, 3]]
    with pytest.raises(ValueError):
        shard.partition_by_cost([1], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SMALL_SIZES = [7, 1, 12, 3, 9, 5, 12, 2, 10, 4]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = shard.partition_by_cost(SMALL_SIZES, world)
        local = {}
        for i in parts[rank]:
            A, B = inputs.base(SMALL_SIZES[i], seed=i)
            om, _, _ = oracle.solve_chol(A, B)
            local[i] = om[: min(3, len(om))]
        merged = shard.gather_to_rank0(local, dist)
        if rank == 0:
            np.save(out_path, np.array([merged[i] for i in range(len(SMALL_SIZES))], dtype=object),
                    allow_pickle=True)
        else:
            assert merged is None
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_shard_and_gather(tmp_path):
    import torch.multiprocessing as mp

    out = str(tmp_path / "merged.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    import oracle

    merged = np.load(out, allow_pickle=True)
    assert len(merged) == len(SMALL_SIZES)
    for i, n in enumerate(SMALL_SIZES):
        A, B = inputs.base(n, seed=i)
        om, _, _ = oracle.solve_chol(A, B)
        assert np.array_equal(merged[i], om[: min(3, n)])
