"""Window sharding across ranks (host logic, CPU): the balanced partition, the ordered
gather of per-window results, and bench.py's max-over-ranks timing, with two `gloo` ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2506_04359_gb300 import shard, synth


def test_partition_is_a_balanced_deterministic_cover():
    cfg = [synth.c3_window_config(s) for s in range(256)]
    costs = [shard.window_cost(c["traj"]["K"], c["M"]) for c in cfg]
    for ws in (1, 2, 3, 8):
        parts = shard.partition(costs, ws)
        assert parts == shard.partition(costs, ws)                   # deterministic
        assert sorted(i for p in parts for i in p) == list(range(256))  # disjoint cover
        loads = [sum(costs[i] for i in p) for p in parts]
        # longest-processing-time bound: max load <= mean + largest single cost
        assert max(loads) <= sum(costs) / ws + max(costs) + 1e-9
    with pytest.raises(ValueError):
        shard.partition(costs, 0)


def test_partition_edge_cases():
    assert shard.partition([], 2) == [[], []]
    assert shard.partition([5.0], 3) == [[0], [], []]
    assert shard.partition([1.0, 1.0, 1.0, 1.0], 2) == [[0, 2], [1, 3]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, costs, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = shard.partition(costs, ws)[rank]
        local = {i: ("rank", rank, i * i) for i in mine}          # stand-in per-window result
        merged = shard.gather(local, ws)
        import bench
        t = bench.max_over_ranks(float(rank + 1), ws)             # the bench's timing reduction
        bench.barrier(ws)
        out.put((rank, sorted(merged.items()), t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_every_window_once():
    costs = [float((7 * i) % 13 + 1) for i in range(40)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = shard.partition(costs, 2)
    for rank, merged, t in res:
        assert [k for k, _ in merged] == list(range(40))
        for k, v in merged:
            assert v[2] == k * k and k in parts[v[1]]
        assert t == 2.0
