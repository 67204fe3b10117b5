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


def test_clock_summary_and_roofline_helpers():
    """Host-side bench helpers: the nvidia-smi sample summary (median clock,
    throttle reasons that were ever active) and the K_bp work model."""
    cs = bench.ClockSampler(0)
    assert cs.summary()["reasons"] == ["unsampled"]
    cs.rows = [["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Active"],
               ["0", "1900", "2070", "950", "0x4", "Not Active", "Active", "Not Active", "Not Active"],
               ["0", "2070", "2070", "880", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0,
                 "reasons": ["hw_thermal_slowdown", "sw_power_cap"], "samples": 3}
    hz, _ = rotated_surface(3)
    h = spacetime(hz, 3)

    class W:
        pass

    w = W()
    w.h = h
    ops, io = bench.roofline_model(w, iters_total=10, shots=4)
    assert ops == 10 * (8 * h.nnz + 2 * h.m + h.n)
    assert io == 4 * (8 * ((h.m + 63) // 64) + 8 * ((h.n + 63) // 64) + 6)
    assert bench.alu_peak_ops(2070.0) == 152 * 128 * 2070e6


def test_roofline_bytes_and_iteration_histogram():
    """The HBM roofline's numerator: B_it = 2 (E b + 4 n) bytes per
    shot-iteration, 544,712 / 364,808 / 274,856 for the d=25 space-time code
    with FP32 / FP16 / INT8 messages (E = 44,976, n = 23,113); and the
    iteration histogram helper (Fig. 6) counts shots per iteration count."""
    from paper_2605_00038_gb300.inputs import workloads
    h = workloads.c5_d25_spacetime(shots=1).h
    assert (h.m, h.n, h.nnz) == (7800, 23113, 44976)
    assert [bench.state_bytes_per_iteration(h, b) for b in (4, 2, 1)] == [544712, 364808, 274856]
    assert bench.io_bytes_per_shot(h) == 8 * 122 + 8 * 362 + 6
    a = torch.tensor([3, 1, 3, 100], dtype=torch.int32)
    b = torch.tensor([100, 100, 7], dtype=torch.int32)
    assert bench.histogram([a, b]) == {"1": 1, "3": 2, "7": 1, "100": 3}
    assert bench.histogram([b, a]) == {"1": 1, "3": 2, "7": 1, "100": 3}


def test_kbp_traffic_names_the_current_kernel_sources():
    """roofline.traffic scales a per-shot-iteration DRAM figure from one ncu
    capture of K_bp; it applies only to the kernel sources it was captured
    from.  The figure, its profile summary and the sources as they stand
    name the same hash: a kernel change without a new capture fails here."""
    from pathlib import Path
    t = bench.KBP_TRAFFIC
    assert t["bytes_per_shot_iteration"] and t["source_sha1"] == bench.kbp_source_sha1()
    prof = (Path(bench.__file__).parent / "profiles" / "bp_ell_kernel_rotated_d25_st25_split.md").read_text()
    assert f"`{t['source_sha1']}`" in prof
    assert f"| DRAM bytes per shot-iteration | {t['bytes_per_shot_iteration']:.1f} " in prof
