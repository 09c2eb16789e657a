"""Host-side logic of the multi-GPU run (no data-path collective), on CPU with gloo and two
ranks: each rank times its own slice groups, the job reports the slowest; the batched job's
items are dealt to the ranks by estimated cost, each item to exactly one rank."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = 100.0 + 50.0 * rank  # rank 1 is the slow replica
    slowest = bench.max_over_ranks(ms)
    # the batched job: each rank takes its own share of the items, then all shares are gathered
    mine = bench.partition_items(bench.item_costs(bench.batched_geometries(), 60), world)[rank]
    shares = [None] * world
    dist.all_gather_object(shares, mine)
    q.put((rank, slowest, bench.seed_for_rank(2, rank), bench.throughput(world, 26, slowest), shares))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_replica_seeds():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]          # both ranks see the slowest time
    assert res[0][2] != res[1][2]                         # replicas draw different slice groups
    assert abs(res[0][3] - 2 * 26 * 1000.0 / 150.0) < 1e-9  # whole-job groups/s
    # every item of the batched job on exactly one rank, and both ranks agree on the split
    shares = res[0][4]
    assert shares == res[1][4]
    flat = sorted(i for sh in shares for i in sh)
    assert flat == list(range(20 * 60))


def test_batched_items_partitioned_by_cost():
    sys.path.insert(0, ROOT)
    import bench

    costs = bench.item_costs(bench.batched_geometries(), 60)
    assert len(costs) == 1200
    for world in (1, 2, 3, 8):
        parts = bench.partition_items(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))  # each item once
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)  # balanced to one item


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.throughput(1, 1, 500.0) == 2.0
