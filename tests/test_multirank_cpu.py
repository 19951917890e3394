"""Multi-rank host logic on CPU: two gloo ranks split independent (poly, limb)
units and ragged items, transform their own share with the oracle, and rank
0 checks that the gathered shares equal the whole batch transformed at once.
Also checks the max-over-ranks timing reduction and the weak-scaling seeds."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2103_16400_gb300 import shard


def test_unit_range_tiles_exactly():
    for n in (0, 1, 5, 31, 32, 33, 1000):
        for world in (1, 2, 3, 8):
            got = [shard.unit_range(n, world, r) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            sizes = [hi - lo for lo, hi in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.unit_range(4, 2, 2)


def test_assign_items_is_a_balanced_partition():
    items = W.ragged_batch(n_polys=64)
    costs = [shard.transform_cost(N, len(qs)) for N, qs in items]
    for world in (1, 2, 4, 8):
        parts = shard.assign_items(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(items)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy longest-first: no rank exceeds the mean by more than the largest item
        assert max(loads) <= sum(costs) / world + max(costs)
    assert shard.assign_items(costs, 3) == shard.assign_items(costs, 3)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # (poly, limb) units of one ciphertext batch
        N = 1024
        moduli = W.mixed_width_primes(5, two_n=2 * N)
        x = W.poly_batch(W.SEED_BASE + 77, 0, 3, moduli, N)
        mine = {}
        for p, l in shard.poly_limb_units(3, len(moduli), world, rank):
            mine[(p, l)] = oracle.ntt_forward_1(x[p, l], moduli[l])
        # ragged items assigned by cost
        items = W.ragged_batch(n_polys=12, log_n_range=(10, 12), max_limbs=3)
        costs = [shard.transform_cost(n, len(qs)) for n, qs in items]
        ragged = {}
        for i in shard.assign_items(costs, world)[rank]:
            n, qs = items[i]
            y = W.poly_batch(W.SEED_BASE + 78, i, 1, qs, n)
            ragged[i] = oracle.ntt_forward(y, qs)
        gathered = [None] * world
        dist.all_gather_object(gathered, (mine, ragged))
        t = shard.max_over_ranks(1.5 + rank)
        if rank == 0:
            units, rag = {}, {}
            for m, r in gathered:
                assert not set(m) & set(units) and not set(r) & set(rag)
                units.update(m)
                rag.update(r)
            full = oracle.ntt_forward(x, moduli)
            assert sorted(units) == [(p, l) for p in range(3) for l in range(len(moduli))]
            for (p, l), v in units.items():
                np.testing.assert_array_equal(v, full[p, l])
            assert sorted(rag) == list(range(len(items)))
            for i, v in rag.items():
                n, qs = items[i]
                y = W.poly_batch(W.SEED_BASE + 78, i, 1, qs, n)
                np.testing.assert_array_equal(v, oracle.ntt_forward(y, qs))
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{t}\n")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        assert float((tmp_path / f"rank{r}.txt").read_text()) == 2.5


def test_rank_seeds_are_distinct():
    seeds = {shard.rank_seed(W.SEED_BASE + 3, r) for r in range(64)}
    assert len(seeds) == 64
    assert shard.rank_seed(5, 0) == 5


def test_max_over_ranks_without_group():
    assert shard.max_over_ranks(3.25) == 3.25
