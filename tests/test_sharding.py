"""The multi-rank path on the CPU: two gloo ranks split the 48-problem sweep by work, each
takes its own share without any data exchange, and the shares (gathered only for the check)
cover every problem exactly once with a makespan within the longest-processing-time bound;
the max-over-ranks reduction of the timings is the one bench.py uses."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from paper_1906_03938_gb300.sharding import shard_by_cost, rank_share


def _costs():
    probs = synth.workload("batch48").problems
    out = []
    for p in probs:
        m = int(p.label.split("_m")[1])
        n = 12 * m * m
        out.append(float(n) * n * p.N)
    return out


def test_shard_by_cost_single_process():
    costs = _costs()
    for world in (1, 2, 3, 4, 8):
        shards = shard_by_cost(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in shards]
        lower = max(sum(costs) / world, max(costs))
        assert max(loads) <= (4.0 / 3.0) * lower + 1e-9 * lower


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = rank_share(costs, rank, world)
    load = torch.tensor([sum(costs[i] for i in mine)], dtype=torch.float64)
    t = load.clone()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)      # the bench's max over ranks
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)         # only for the check
    if rank == 0:
        out.put((gathered, float(t[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_without_exchange():
    costs = _costs()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(i for s in gathered for i in s)
    assert flat == list(range(len(costs)))
    assert set(gathered[0]).isdisjoint(gathered[1])
    loads = [sum(costs[i] for i in s) for s in gathered]
    assert tmax == max(loads)
    assert max(loads) <= (4.0 / 3.0) * max(sum(costs) / world, max(costs))
