"""The multi-rank path of bench.py on CPU: two gloo ranks shard the workload's configurations
(disjoint, covering), take the max of their times and aggregate the rate like bench.py does."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import fd_inputs as fi
    from paper_2604_02130_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    per = 6
    idx = list(shard.shard_range(rank, per))
    probs = fi.workload("batch18", batch=per, first=idx[0])
    # the first field value of every configuration identifies it
    mine = torch.tensor([p.phi[0, 0] for p in probs], dtype=torch.float64)
    gathered = [torch.zeros(per, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, mine)
    t = shard.max_over_ranks(10.0 + rank)
    rate = shard.aggregate_rate(per, world, steps=3, max_ms=t)
    if rank == 0:
        out.put((torch.cat(gathered).numpy(), t, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_are_disjoint_and_time_is_max():
    import multiprocessing as mp

    import fd_inputs as fi

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    firsts, t, rate = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = np.array([p.phi[0, 0] for p in fi.workload("batch18", batch=12)])
    assert np.array_equal(firsts, ref)          # rank 0 took 0..5, rank 1 took 6..11
    assert t == 11.0                            # max over ranks
    assert abs(rate - 12 * 3 / 11e-3) < 1e-9    # all configurations over the slowest rank


def test_lpt_partition_balances_costs():
    from paper_2604_02130_gb300 import shard

    costs = [7.0, 5.0, 4.0, 3.0, 3.0, 2.0]
    parts = shard.lpt_partition(costs, 2)
    assert sorted(parts[0] + parts[1]) == list(range(6))
    # LPT: 7 -> r0, 5 -> r1, 4 -> r1, 3 -> r0, 3 -> r0 (10 vs 9: r1), ... = loads 12 and 12
    loads = [sum(costs[i] for i in p) for p in parts]
    assert loads == [12.0, 12.0]
    assert shard.lpt_partition([1.0], 3) == [[0], [], []]


def _rank_uneven(rank, world, port, out):
    import torch.distributed as dist

    import fd_inputs as fi
    from paper_2604_02130_gb300 import shard

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    per = 512
    sizes = fi.uneven_sizes(per * world)
    costs = [(2 * L * L) ** 3 * nt for (L, nt) in sizes]
    mine = shard.lpt_partition(costs, world)[rank]
    t = torch.zeros(per * world, dtype=torch.int64)
    t[mine] = rank + 1
    dist.all_reduce(t)  # each index owned once: the sum over ranks is its owner + 1
    load = torch.tensor([float(sum(costs[i] for i in mine))], dtype=torch.float64)
    loads = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(loads, load)
    if rank == 0:
        out.put((t.numpy(), [float(x) for x in loads], len(mine)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_uneven_shards_are_cost_balanced():
    """The uneven workload's two-rank split (bench.py): every configuration index once, and the
    ranks' Nx^3 Nt totals within 1 % of each other."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + ((os.getpid() + 500) % 1000)
    procs = [ctx.Process(target=_rank_uneven, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    owner, loads, n0 = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert set(np.unique(owner)) == {1, 2} and owner.min() >= 1
    assert max(loads) / min(loads) < 1.01
    assert 400 < n0 < 624
