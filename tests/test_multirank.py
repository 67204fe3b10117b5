"""The N > 1 path of the benchmark on CPU with two gloo ranks: ranks decode
disjoint shot ranges keyed by global shot index (no data-path collective), and
the job's value uses the maximum time over ranks."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2605_00038_gb300.inputs import sampler
from paper_2605_00038_gb300.inputs.codes import rotated_surface, spacetime, spacetime_priors


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, shots, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    offs = bench.rank_offsets(rank, shots)
    hz, _ = rotated_surface(3)
    h = spacetime(hz, 3)
    pri = spacetime_priors(hz, 3, 0.02, 0.02)
    _, syn = sampler.sample(h, pri, seed=5, num_shots=shots, shot_offset=offs[1])
    elapsed = 10.0 * (rank + 1)                      # rank 1 is the slow one
    max_ms, value = bench.job_value(world, shots, 4, elapsed, dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, offs)
    dist.destroy_process_group()
    q.put((rank, offs, syn, max_ms, value, gathered))


def test_two_gloo_ranks_split_shots_and_take_max_time():
    world, shots = 2, 64
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, shots, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=120) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ranges = set()
    for rank, offs, syn, max_ms, value, gathered in res:
        assert max_ms == 20.0
        assert value == world * shots * 4 / 0.020
        for o in offs:
            ranges.add((o, o + shots))
    assert len(ranges) == world * bench.N_BATCHES
    spans = sorted(ranges)
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    # A rank's batch is exactly the global shots it is keyed by.
    hz, _ = rotated_surface(3)
    h = spacetime(hz, 3)
    pri = spacetime_priors(hz, 3, 0.02, 0.02)
    r1 = res[1]
    _, full = sampler.sample(h, pri, seed=5, num_shots=r1[1][1] + shots)
    assert np.array_equal(full[r1[1][1]:], r1[2])
