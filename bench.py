#!/usr/bin/env python3
"""Throughput benchmark of the Lottery BP + OSD-0 decoder on GB300.

One step = one pass of the whole decoding path (BP with the lottery on every
shot, OSD-0 on the shots BP leaves unconverged) over one batch of seeded
synthetic syndromes of the rotated d=11 surface code with 11 noisy rounds
(space-time H 660 x 1931, nnz 3620), p_data = p_meas = 0.003, 10^6 shots,
max 100 iterations, binary32 messages.

Prints one JSON line (rank 0).  `value` is decoded shots per second over all
ranks with inputs resident in HBM; `e2e` is the same through the host-buffer
entry point with the copies inside the timed region.  `--impl reference`
times the CPU oracle instead (on a bounded sample of the same workload).
Under torchrun each rank decodes its own shots (weak scaling; no data-path
collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "decoded shots/sec and p99 decode latency at matched logical error rate; HBM GB/s"
UNIT = "shots/s"
N_BATCHES = 3        # rotating input batches: 3 x 88 MB of syndromes > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--shots", type=int, default=1_000_000, help="shots per step per rank")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip latency sweep, LER and CPU baseline")
    ap.add_argument("--cpu-sample", type=int, default=20_000, help="oracle shots for cpu_baseline")
    ap.add_argument("--no-tune", action="store_true", help="skip lbp_tune (default launch shape)")
    ap.add_argument("--serving-only", action="store_true", help="print the serving and matched-LER results only")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ---------------------------------------------------------------- helpers

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_offsets(rank: int, shots: int, n_batches: int = N_BATCHES):
    """Global index of shot 0 of each input batch of `rank`: ranks decode
    disjoint shot ranges, keyed by global index (weak scaling)."""
    return [(rank * n_batches + k) * shots for k in range(n_batches)]


def job_value(world: int, shots: int, steps: int, elapsed_ms_per_rank, dist=None):
    """(max elapsed ms over ranks, whole-job shots/s).  `elapsed_ms_per_rank`
    is this rank's time; with a process group the max is all-reduced."""
    import torch
    t = torch.tensor([float(elapsed_ms_per_rank)],
                     device="cuda" if (dist is not None and dist.get_backend() == "nccl") else "cpu")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    max_ms = float(t.item())
    return max_ms, world * shots * steps / (max_ms / 1e3)


def workload(shots):
    from paper_2605_00038_gb300.inputs import workloads
    return workloads.c2_d11_spacetime(shots=shots, osd=1)


def roofline_model(w, iters_total, shots):
    """Algorithmic work of K_bp: per shot-iteration 8 E + 2 m + n operations
    (per edge the V2C subtract, two minimum compares, sign parity, output
    select and sign, LLR add and syndrome XOR; per check two scale multiplies;
    per column the hard decision); per shot the syndrome in and results out."""
    E, m, n = w.h.nnz, w.h.m, w.h.n
    ops = float(iters_total) * (8 * E + 2 * m + n)
    io = shots * (8 * ((m + 63) // 64) + 8 * ((n + 63) // 64) + 1 + 1 + 4)
    return ops, io


# DRAM bytes per shot of K_bp on this workload (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture, 131,072 shots, scaled per shot),
# valid for the kernel sources whose hash is recorded with it.
KBP_TRAFFIC = {"bytes_per_shot": 1135.5, "source_sha1": "e49ad615ca0e"}


def kbp_source_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in ("bp_ell_kernel.cuh", "bp_common.cuh", "bp_graph.cuh"):
        h.update((ROOT / "paper_2605_00038_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:12]


def alu_peak_ops(sm_mhz):
    # 152 SMs x 4 sub-partitions x 32 lanes, one instruction per lane per clock.
    return 152 * 4 * 32 * sm_mhz * 1e6


# ------------------------------------------------------------- reference arm

def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    from paper_2605_00038_gb300.inputs import sampler
    w = workload(args.shots)
    cores = os.cpu_count() or 1
    sample = max(1, min(args.cpu_sample, w.shots))
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=sample)
    S = sampler.unpack(syn, w.h.m)
    prm = oracle.OracleParams(max_iter=100, lottery=True, lottery_skip=6, osd=True,
                              prec=oracle.PREC_F64, seed=w.seed)
    for _ in range(args.warmup):
        oracle.decode(w.h, w.priors, S[: max(1, sample // 20)], prm, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.decode(w.h, w.priors, S, prm, nthreads=cores)
    dt = time.perf_counter() - t0
    v = sample * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "shots_per_step": sample, "decoder": "lottery_bp+osd0",
                   "max_iter": 100, "parallelism": "cpu threads"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d shots of %s per step (FP64 oracle, %d threads)"
                                   % (sample, w.name, cores)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def logical_failures(w, err_words, est_words, conv, osd):
    """Logical failure per shot: the residual's data part, summed over rounds,
    hits a logical operator; or BP did not converge and OSD did not apply."""
    import torch
    from paper_2605_00038_gb300.inputs.codes import logical_operators, rotated_surface
    hz, hx = rotated_surface(11)
    L = torch.from_numpy(logical_operators(hz, hx).astype(np.float32)).cuda()
    T, nq = 11, hz.n
    fails = 0
    B = err_words.shape[0]
    shifts = torch.arange(64, device="cuda", dtype=torch.int64)
    for lo in range(0, B, 50_000):
        r = torch.bitwise_xor(err_words[lo:lo + 50_000], est_words[lo:lo + 50_000])
        bits = torch.bitwise_and(torch.bitwise_right_shift(r.unsqueeze(-1), shifts), 1)
        bits = bits.reshape(r.shape[0], -1)[:, : w.h.n]
        data = bits[:, : T * nq].reshape(-1, T, nq).sum(1).remainder(2).float()
        hit = (data @ L.T).remainder(2).sum(1) > 0
        bad = (conv[lo:lo + 50_000] == 0) & (osd[lo:lo + 50_000] != 1)
        fails += int((hit | bad).sum().item())
    return fails


def run_gpu(args):
    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_00038_gb300 import lbp
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler

    w = workload(args.shots)
    B = w.shots
    dec = Decoder(w.h, w.priors, device="cuda:%d" % local)
    wm, wn = (w.h.m + 63) // 64, (w.h.n + 63) // 64

    # Inputs: N_BATCHES distinct batches per rank, resident on the device.
    syn_h, err_h, syn_d, prms = [], [], [], []
    for k, off in enumerate(rank_offsets(rank, B)):
        e, s = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=B, shot_offset=off)
        err_h.append(e)
        syn_h.append(s)
        syn_d.append(torch.from_numpy(s.view(np.int64)).cuda())
        prms.append(dec.params(**w.decoder, seed=w.seed, shot_offset=off))
    outs = [dec.alloc(B) for _ in range(N_BATCHES)]
    ws = dec.workspace(prms[0], B)
    stream = torch.cuda.current_stream()

    def step(k):
        lbp.lbp_decode(dec.code, prms[k % N_BATCHES], B, syn_d[k % N_BATCHES], outs[k % N_BATCHES].err,
                       outs[k % N_BATCHES].converged, outs[k % N_BATCHES].osd,
                       outs[k % N_BATCHES].iters, None, ws, stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # Launch-shape autotuning on the first batch (outside the timed region).
    launch = None
    if not args.no_tune:
        tb = min(B, 131072)
        dec.tune(syn_d[0][:tb].contiguous(), prms[0], stream)
        S_t, G_t, gf_t = lbp.lbp_code_tuned(dec.code, prms[0].msg, prms[0].rule)
        launch = {"groups_per_cta": S_t, "threads_per_shot": G_t,
                  "graph": {0: "default", 1: "index image", 2: "implicit", 3: "round"}.get(gf_t, str(gf_t))}
    for k in range(args.warmup):
        step(k)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    lbp.lbp_timing_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(stream)
    for k in range(args.steps):
        step(k)
    ev1.record(stream)
    barrier()
    clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    bp_ms, bp_n, osd_ms, osd_n = lbp.lbp_timing_read()
    lbp.lbp_timing_enable(False)
    max_ms, value = job_value(world, B, args.steps, elapsed_ms, dist)

    # Work actually done in the timed steps (iterations, OSD invocations).
    iters_total = 0
    osd_total = 0
    for k in range(args.steps):
        o = outs[k % N_BATCHES]
        iters_total += int(o.iters.sum().item())
        osd_total += int((o.osd != 0).sum().item())

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "code": "rotated surface d=11, 11 rounds, H_st 660x1931 nnz 3620",
                   "noise": "iid p_data=p_meas=0.003", "shots_per_step_per_rank": B,
                   "decoder": "lottery_bp(skip 6, adaptive scale, I=100) + osd0",
                   "msg": "f32", "l2": "3 rotating input batches (%d MB syndromes) > L2" % (
                       N_BATCHES * B * wm * 8 // 2 ** 20),
                   "parallelism": "replicas" if world > 1 else "single"},
        "clocks": clocks.summary(),
        "gpu_launches": int(bp_n + osd_n),
    }
    sm_mhz = line["clocks"]["sm_mhz"] or 2070.0
    ops, io = roofline_model(w, iters_total / args.steps, B)
    bp_avg_s = bp_ms / max(bp_n, 1) / 1e3
    peak = alu_peak_ops(sm_mhz)
    traffic = (KBP_TRAFFIC["bytes_per_shot"] * B
               if kbp_source_sha1() == KBP_TRAFFIC["source_sha1"] else None)
    # Shared-memory view: per shot-iteration the state the algorithm must move
    # (read lambda and beta, write beta on each edge; read beta per edge and
    # write lambda per column), E (4 + 3b) + 8 n bytes, against
    # 152 SMs x 128 B/clock.
    E, n = w.h.nnz, w.h.n
    smem_bytes = (iters_total / args.steps) * (E * (4 + 3 * 4) + 8 * n)
    smem_peak = 152 * 128 * sm_mhz * 1e6
    line["roofline"] = {"bound": "alu", "achieved": ops / bp_avg_s / 1e12, "peak": peak / 1e12,
                        "unit": "Tops/s", "frac": (ops / bp_avg_s) / peak, "traffic": traffic,
                        "kernel": "bp_ell_kernel", "avg_launch_ms": bp_avg_s * 1e3,
                        "ops_per_launch": ops, "io_bytes_per_launch": io,
                        "dram_gbs_from_traffic": (traffic / bp_avg_s / 1e9) if traffic else None,
                        "peak_basis": "152 SMs x 128 lanes x median SM clock %.0f MHz (derived)" % sm_mhz,
                        "smem": {"achieved_tbs": smem_bytes / bp_avg_s / 1e12,
                                 "peak_tbs": smem_peak / 1e12,
                                 "frac": smem_bytes / bp_avg_s / smem_peak,
                                 "note": "per ncu: shared-memory pipe 85% busy and instruction issue "
                                         "77%; 30% of load wavefronts bank conflicts"}}
    line["kernels"] = {"bp_launch": launch, "bp_ms_per_step": bp_ms / args.steps,
                       "osd_ms_per_step": osd_ms / args.steps,
                       "mean_iters": iters_total / (B * args.steps),
                       "osd_invoke_rate": osd_total / (B * args.steps)}

    # End to end through the host-buffer entry point (pinned memory).
    if not args.no_e2e:
        pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()
        hs = []
        for k in range(N_BATCHES):
            p = pin(syn_h[k].shape, torch.int64)
            p.numpy()[:] = syn_h[k].view(np.int64)
            hs.append(p)
        ho = dict(err=pin((B, wn), torch.int64), converged=pin(B, torch.uint8), osd=pin(B, torch.uint8),
                  iters=pin(B, torch.int32))
        hws = dec.workspace(prms[0], B, host=True)

        def hstep(k):
            lbp.lbp_decode_host(dec.code, prms[k % N_BATCHES], B, hs[k % N_BATCHES], ho["err"],
                                ho["converged"], ho["osd"], ho["iters"], None, hws, stream)

        hstep(0)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            hstep(k)
        e1.record(stream)
        barrier()
        _, e2e_value = job_value(world, B, args.steps, e0.elapsed_time(e1), dist)
        line["e2e"] = {"value": e2e_value, "unit": UNIT,
                       "h2d_bytes_per_step": B * wm * 8,
                       "d2h_bytes_per_step": B * (wn * 8 + 1 + 1 + 4)}

    if not args.no_extras and rank == 0:
        # Per-batch latency at small batch sizes (outside the timed region):
        # each repeat decodes different shots of batch 0, so the quantiles are
        # over the workload's shots (converged and OSD-bound alike), not over
        # timing jitter of one batch.
        lat = {}
        for bs, reps in ((1, 210), (64, 210), (4096, 60)):
            o = dec.alloc(bs)
            wsb = dec.workspace(prms[0], bs)
            times = []
            for r in range(reps):
                lo = (r * bs) % max(1, B - bs + 1)
                sub = syn_d[0][lo:lo + bs].contiguous()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lbp.lbp_decode(dec.code, prms[0], bs, sub, o.err, o.converged, o.osd, o.iters, None,
                               wsb, stream)
                b.record(stream)
                b.synchronize()
                if r >= 10:
                    times.append(a.elapsed_time(b))
            times.sort()
            lat["batch_%d" % bs] = {"p50_ms": times[len(times) // 2],
                                    "p99_ms": times[min(len(times) - 1, int(0.99 * len(times)))],
                                    "samples": len(times)}
        # Batch 1 replayed from a CUDA graph (lbp_graph_*): the same decode
        # without the per-call cost of issuing its stream operations.  Each
        # repeat first writes a different shot into the captured buffer.
        x1 = torch.empty((1, wm), dtype=torch.int64, device=syn_d[0].device)
        o1 = dec.alloc(1)
        ws1 = torch.empty(lbp.lbp_workspace_size(dec.code, prms[0], 1) + 256, dtype=torch.uint8,
                          device=syn_d[0].device)
        ws1 = ws1[(-ws1.data_ptr()) % 256:]
        g1 = lbp.lbp_graph_create(dec.code, prms[0], 1, x1, o1.err, o1.converged, o1.osd, o1.iters, None,
                                  ws1)
        times = []
        for r in range(210):
            x1.copy_(syn_d[0][r:r + 1])
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lbp.lbp_graph_launch(g1, stream)
            b.record(stream)
            b.synchronize()
            if r >= 10:
                times.append(a.elapsed_time(b))
        g1.close()
        times.sort()
        lat["batch_1_graph"] = {"p50_ms": times[len(times) // 2],
                                "p99_ms": times[min(len(times) - 1, int(0.99 * len(times)))],
                                "samples": len(times)}
        lat["batch_%d" % B] = {"p50_ms": line["ms_per_step"], "p99_ms": None}
        line["latency"] = lat
        # Logical error rate of batch 0 (true errors known from the sampler).
        o = outs[0]
        step(0)
        torch.cuda.synchronize()
        fails = logical_failures(w, torch.from_numpy(err_h[0].view(np.int64)).cuda(), o.err,
                                 o.converged, o.osd)
        line["quality"] = {"ler": fails / B, "shots": B, "logical_failures": fails}

    if not args.no_extras and rank == 0 and world == 1:
        line["serving"] = run_serving()
        line["serving_one_launch_fifo"] = run_serving(policy=(0, False))
        line["matched_ler"] = run_matched()
        line["precision"] = run_precision()
        line["lottery_design_space"] = run_policies()
        line["check_rule"] = run_sum_product()
    if not args.no_extras and rank == 0 and world == 1:
        import oracle
        cores = os.cpu_count() or 1
        S = sampler.unpack(syn_h[0][: args.cpu_sample], w.h.m)
        prm = oracle.OracleParams(max_iter=100, lottery=True, lottery_skip=6, osd=True,
                                  prec=oracle.PREC_F64, seed=w.seed, shot_offset=0)
        t0 = time.perf_counter()
        oracle.decode(w.h, w.priors, S, prm, nthreads=cores)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": S.shape[0] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%d shots of %s (FP64 oracle, %d threads, %.1f s)"
                                          % (S.shape[0], w.name, cores, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    dec.close()
    if dist is not None:
        dist.destroy_process_group()


def run_serving(seconds_per_rate: float = 3.0, n_requests: int = 600, seed: int = 11, policy=None):
    """Serving mix: Poisson arrivals of 1-4096-shot requests over ten resident
    codes (rotated surface space-time d = 5..17 with d rounds, BB 72/144/288
    code capacity) and five noise levels 1e-3..5e-3; Lottery BP + OSD-0,
    I = 100, INT8 messages.  Capacity first (all requests queued at once), then
    open-loop arrivals at 50 / 80 / 95 % of it.  Messages are Int3.4 (INT8),
    the format the paper's hardware uses; FP16 messages roughly double the
    lottery's OSD invoke rate on these surface codes.  policy: None for the
    server's default scheduling (launches of at most 16 Mi edge-shots,
    single-launch requests on a high-priority stream), or (chunk_work,
    priority) for lbp_server_configure."""
    import torch
    from paper_2605_00038_gb300 import lbp
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler, workloads
    from paper_2605_00038_gb300.inputs.codes import spacetime_priors

    ps = (0.001, 0.002, 0.003, 0.004, 0.005)
    codes = workloads.serving_codes()
    decs = {}
    rounds = {}
    for ci, (name, h, st_info) in enumerate(codes):
        for pi, p in enumerate(ps):
            if st_info is not None:
                hz, d = st_info
                pri = spacetime_priors(hz, d, p, p)
                rounds[ci] = d
            else:
                pri = np.full(h.n, p)
                rounds[ci] = 1
            decs[(ci, pi)] = Decoder(h, pri)
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n_requests):
        ci, pi = int(rng.integers(len(codes))), int(rng.integers(len(ps)))
        B = int(round(np.exp(rng.uniform(0, np.log(4096)))))
        dec = decs[(ci, pi)]
        h = dec.h
        _, syn = sampler.sample(h, dec_priors(dec), seed=seed + ci, num_shots=B, shot_offset=i << 16)
        pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()
        s = pin(syn.shape, torch.int64)
        s.numpy()[:] = syn.view(np.int64)
        reqs.append(dict(ci=ci, pi=pi, B=B, syn=s, err=pin((B, (h.n + 63) // 64), torch.int64),
                         conv=pin(B, torch.uint8), osd=pin(B, torch.uint8), iters=pin(B, torch.int32),
                         prm=dec.params(max_iter=100, lottery=1, osd=1, msg=2, seed=seed,
                                        shot_offset=i << 16)))
    srv = lbp.lbp_server_create(8 << 30, 16)
    if policy is not None:
        lbp.lbp_server_configure(srv, policy[0], policy[1])

    def submit(r):
        return lbp.lbp_server_submit(srv, decs[(r["ci"], r["pi"])].code, r["prm"], r["B"], r["syn"],
                                     r["err"], r["conv"], r["osd"], r["iters"])

    # warm-up: one request per code / noise pair
    for k in range(min(len(reqs), 50)):
        lbp.lbp_server_wait(srv, submit(reqs[k]))
    t0 = time.perf_counter()
    tickets = [submit(r) for r in reqs]
    for t in tickets:
        lbp.lbp_server_wait(srv, t)
    dt = time.perf_counter() - t0
    total_shots = sum(r["B"] for r in reqs)
    cap_req = len(reqs) / dt
    out = {"policy": ("chunk_work 16 Mi edge-shots, priority" if policy is None else
                      "chunk_work %d, priority %d" % (policy[0], int(policy[1]))),
           "codes": len(codes), "noise_levels": len(ps), "requests": len(reqs),
           "mean_request_shots": total_shots / len(reqs), "capacity_shots_per_s": total_shots / dt,
           "capacity_requests_per_s": cap_req, "rates": []}
    for load in (0.5, 0.8, 0.95):
        rate = load * cap_req
        n = max(20, min(len(reqs), int(rate * seconds_per_rate)))
        gaps = rng.exponential(1.0 / rate, size=n)
        order = rng.permutation(len(reqs))[:n]
        sent = []
        t_start = time.perf_counter()
        t_next = t_start
        for j, i in enumerate(order):
            t_next += gaps[j]
            while True:
                now = time.perf_counter()
                if now >= t_next:
                    break
                time.sleep(min(0.0005, t_next - now))
            sent.append((i, submit(reqs[i])))
        lats, per_round = [], []
        for i, t in sent:
            lat = lbp.lbp_server_wait(srv, t)
            lats.append(lat)
            per_round.append(lat / rounds[reqs[i]["ci"]])
        span = time.perf_counter() - t_start
        q = lambda a, x: float(np.quantile(np.asarray(a), x) * 1e3)
        out["rates"].append({"load": load, "offered_requests_per_s": rate, "requests": n,
                             "shots_per_s": sum(reqs[i]["B"] for i, _ in sent) / span,
                             "p50_ms": q(lats, 0.5), "p99_ms": q(lats, 0.99),
                             "p50_ms_per_round": q(per_round, 0.5), "p99_ms_per_round": q(per_round, 0.99)})
    srv.close()
    for d in decs.values():
        d.close()
    return out


def dec_priors(dec):
    return dec.priors


def run_matched(shots: int = 1 << 20, request: int = 4096, seed: int = 21):
    """Matched-LER head-to-head on identical shots of the rotated d=7 surface
    code, 7 noisy rounds, p = 0.012: (A) plain NMS BP + OSD-0, FP32 messages,
    one batched lbp_decode; (B) Lottery BP + OSD-0, INT8 (Int3.4) messages, served in
    4096-shot requests through lbp_server, with the proposed flip rule and
    with the worst-check / least-reliable-column rule of Sec. III-B.  Logical
    error rates with Wilson 95% intervals and the paired McNemar test against
    (A), throughput and p50 / p99 request latency."""
    import torch
    from paper_2605_00038_gb300 import evaluate, lbp
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler
    from paper_2605_00038_gb300.inputs.codes import rotated_surface, spacetime, spacetime_priors

    d, p = 7, 0.012
    hz, _ = rotated_surface(d)
    h = spacetime(hz, d)
    pri = spacetime_priors(hz, d, p, p)
    e, syn = sampler.sample(h, pri, seed=seed, num_shots=shots)
    spec = evaluate.surface_spec(d, d, h.n)
    true_d = torch.from_numpy(e.view(np.int64)).cuda()
    dec = Decoder(h, pri)
    # Arm A: plain BP + OSD-0, FP32, batched.
    pa = dec.params(max_iter=100, lottery=0, osd=1, msg=0, seed=seed)
    sd = torch.from_numpy(syn.view(np.int64)).cuda()
    dec.decode(sd, pa)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    ra = dec.decode(sd, pa)
    ev1.record()
    torch.cuda.synchronize()
    ta = ev0.elapsed_time(ev1) / 1e3
    fa = evaluate.logical_failures(spec, true_d, ra.err, ra.converged, ra.osd)
    ka = int(fa.sum().item())
    out = {
        "workload": "rotated_d7_st7_p0.012", "shots": shots,
        "plain_bp_osd_fp32_batched": {
            "ler": ka / shots, "ler_ci95": evaluate.wilson(ka, shots), "shots_per_s": shots / ta,
            "latency_ms": ta * 1e3, "osd_invoke_rate": float((ra.osd != 0).float().mean().item()),
            "mean_iters": float(ra.iters.float().mean().item())},
    }
    # Arms B: Lottery BP + OSD-0, INT8, served.
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()
    hs = pin(syn.shape, torch.int64)
    hs.numpy()[:] = syn.view(np.int64)
    wn = (h.n + 63) // 64
    herr, hconv, hosd, hit = pin((shots, wn), torch.int64), pin(shots, torch.uint8), pin(shots, torch.uint8), pin(shots, torch.int32)
    for key, policy in (("lottery_bp_osd_int8_served", lbp.LBP_LOTTERY_PROPOSED),
                        ("lottery_worst_unreliable_bp_osd_int8_served", lbp.LBP_LOTTERY_WORST_UNRELIABLE)):
        srv = lbp.lbp_server_create(8 << 30, 16)
        reqs = []
        for lo in range(0, shots, request):
            B = min(request, shots - lo)
            prm = dec.params(max_iter=100, lottery=1, lottery_policy=policy, osd=1, msg=2, seed=seed,
                             shot_offset=lo)
            reqs.append((lo, B, prm))
        lbp.lbp_server_wait(srv, lbp.lbp_server_submit(srv, dec.code, reqs[0][2], reqs[0][1], hs[:reqs[0][1]],
                                                       herr[:reqs[0][1]], hconv[:reqs[0][1]],
                                                       hosd[:reqs[0][1]], hit[:reqs[0][1]]))
        t0 = time.perf_counter()
        tks = [lbp.lbp_server_submit(srv, dec.code, prm, B, hs[lo:lo + B], herr[lo:lo + B], hconv[lo:lo + B],
                                     hosd[lo:lo + B], hit[lo:lo + B]) for lo, B, prm in reqs]
        lats = [lbp.lbp_server_wait(srv, t) for t in tks]
        tb = time.perf_counter() - t0
        srv.close()
        fb = evaluate.logical_failures(spec, true_d, herr.cuda(), hconv.cuda(), hosd.cuda())
        kb = int(fb.sum().item())
        only_a = int((fa & ~fb).sum().item())
        only_b = int((fb & ~fa).sum().item())
        out[key] = {
            "policy": policy, "ler": kb / shots, "ler_ci95": evaluate.wilson(kb, shots),
            "shots_per_s": shots / tb, "request_shots": request,
            "p50_ms": float(np.quantile(lats, 0.5) * 1e3), "p99_ms": float(np.quantile(lats, 0.99) * 1e3),
            "osd_invoke_rate": float((hosd != 0).float().mean().item()),
            "mean_iters": float(hit.float().mean().item()),
            "ler_relative_difference": (kb - ka) / max(ka, 1), "mcnemar_discordant": [only_a, only_b],
            "mcnemar_p": evaluate.mcnemar_p(only_a, only_b)}
    dec.close()
    return out


def run_precision(shots: int = 1 << 20, oracle_shots: int = 1 << 15, seed: int = 31):
    """Precision gap: Lottery BP + OSD-0 on the rotated d=7 surface code, 7
    noisy rounds, p = 0.012, with FP32 / FP16 / INT8 messages (2^20 shots
    each, identical shots), against the FP64 oracle on the first 2^15 shots.
    Then throughput of the d=25, 25-round code (7,800 x 23,113) per precision."""
    import torch
    import oracle
    from paper_2605_00038_gb300 import evaluate
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler, workloads
    from paper_2605_00038_gb300.inputs.codes import rotated_surface, spacetime, spacetime_priors

    d, p = 7, 0.012
    hz, _ = rotated_surface(d)
    h = spacetime(hz, d)
    pri = spacetime_priors(hz, d, p, p)
    e, syn = sampler.sample(h, pri, seed=seed, num_shots=shots)
    spec = evaluate.surface_spec(d, d, h.n)
    true_d = torch.from_numpy(e.view(np.int64)).cuda()
    sd = torch.from_numpy(syn.view(np.int64)).cuda()
    dec = Decoder(h, pri)
    cores = os.cpu_count() or 1
    r = oracle.decode(h, pri, sampler.unpack(syn[:oracle_shots], h.m),
                      oracle.OracleParams(max_iter=100, lottery=True, osd=True, prec=oracle.PREC_F64,
                                          seed=seed), nthreads=cores)
    fo = evaluate.logical_failures(spec, true_d[:oracle_shots].cpu(),
                                   torch.from_numpy(sampler.pack(r.err).view(np.int64)),
                                   torch.from_numpy(r.converged), torch.from_numpy(r.osd_used)).numpy()
    out = {"workload": "rotated_d7_st7_p0.012", "shots": shots, "oracle_shots": oracle_shots,
           "fp64_oracle": {"ler_subset": float(fo.mean()), "osd_invoke_rate_subset": float(r.osd_used.mean())}}
    for msg, name in ((0, "fp32"), (1, "fp16"), (2, "int8")):
        prm = dec.params(max_iter=100, lottery=1, osd=1, msg=msg, seed=seed)
        res = dec.decode(sd, prm)
        torch.cuda.synchronize()
        f = evaluate.logical_failures(spec, true_d, res.err, res.converged, res.osd).cpu().numpy()
        fs = f[:oracle_shots]
        k = int(f.sum())
        out[name] = {"ler": k / shots, "ler_ci95": evaluate.wilson(k, shots),
                     "ler_subset": float(fs.mean()),
                     "gap_vs_fp64_subset": float(fs.mean() - fo.mean()),
                     "mcnemar_p_vs_fp64": evaluate.mcnemar_p(int((fs & ~fo).sum()), int((fo & ~fs).sum())),
                     "osd_invoke_rate": float((res.osd != 0).float().mean().item()),
                     "mean_iters": float(res.iters.float().mean().item())}
    dec.close()
    # d=25 throughput per precision (no OSD, as configured).
    c5 = {}
    for msg, name in ((0, "fp32"), (1, "fp16"), (2, "int8")):
        w = workloads.c5_d25_spacetime(msg=msg, shots=1 << 17)
        _, s5 = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
        d5 = Decoder(w.h, w.priors)
        prm = d5.params(**w.decoder)
        s5d = torch.from_numpy(s5.view(np.int64)).cuda()
        d5.tune(s5d[:16384].contiguous(), prm)
        d5.decode(s5d, prm)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        res = d5.decode(s5d, prm)
        a1.record()
        torch.cuda.synchronize()
        t = a0.elapsed_time(a1) / 1e3
        it = float(res.iters.float().mean().item())
        bpm = {0: 4, 1: 2, 2: 1}[msg]
        c5[name] = {"shots_per_s": w.shots / t, "mean_iters": it,
                    "unconverged": float((res.converged == 0).float().mean().item()),
                    "state_gbs": w.shots * it * 2 * (w.h.nnz * bpm + 4 * w.h.n) / t / 1e9}
        d5.close()
    out["d25_throughput"] = c5
    # d=27 in the form of Table II (unrotated code, cyclic boundary, 18,954 x
    # 56,889): the paper's simulator ran out of GPU memory here.
    from paper_2605_00038_gb300.inputs.codes import unrotated_surface
    _, hz27 = unrotated_surface(27)
    st27 = spacetime(hz27, 27, "cyclic")
    pri27 = np.full(st27.n, 0.004)
    d27 = Decoder(st27, pri27)
    n27 = 1 << 13
    _, s27 = sampler.sample(st27, pri27, seed=27, num_shots=n27)
    s27d = torch.from_numpy(s27.view(np.int64)).cuda()
    prm = d27.params(max_iter=100, lottery=1, osd=0, msg=0, seed=27)
    d27.decode(s27d[:512].contiguous(), prm)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record()
    res = d27.decode(s27d, prm)
    a1.record()
    torch.cuda.synchronize()
    t = a0.elapsed_time(a1) / 1e3
    out["d27_table2_fp32"] = {"shape": [st27.m, st27.n, st27.nnz], "shots": n27, "shots_per_s": n27 / t,
                              "mean_iters": float(res.iters.float().mean().item()),
                              "device_state_mb_per_shot": (6 * (st27.m + 3) * 4 + 4 * (st27.n + 3)) / 2 ** 20}
    d27.close()
    return out


def run_policies(shots: int = 1 << 18, seed: int = 41):
    """Lottery design space (Sec. III-B, Table I, Fig. 5) on the rotated d=9
    surface code with 9 noisy rounds, p = 0.005, FP32, I = 100: logical error
    rate of BP alone (unconverged shots count as failures) and OSD invoke
    rate, for plain BP, the proposed policy and the four baselines (skip 6),
    then the proposed policy's skip-iteration sweep."""
    import torch
    from paper_2605_00038_gb300 import evaluate
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler
    from paper_2605_00038_gb300.inputs.codes import rotated_surface, spacetime, spacetime_priors

    d, p = 9, 0.005
    hz, _ = rotated_surface(d)
    h = spacetime(hz, d)
    pri = spacetime_priors(hz, d, p, p)
    e, syn = sampler.sample(h, pri, seed=seed, num_shots=shots)
    spec = evaluate.surface_spec(d, d, h.n)
    true_d = torch.from_numpy(e.view(np.int64)).cuda()
    sd = torch.from_numpy(syn.view(np.int64)).cuda()
    dec = Decoder(h, pri)
    names = {0: "proposed", 1: "worst_cn_unreliable_vn", 2: "worst_cn_random_vn",
             3: "random_cn_unreliable_vn", 4: "random_cn_random_vn"}

    def one(**kw):
        r = dec.decode(sd, dec.params(max_iter=100, osd=0, msg=0, seed=seed, **kw))
        torch.cuda.synchronize()
        f = evaluate.logical_failures(spec, true_d, r.err, r.converged, r.osd)
        k = int(f.sum().item())
        return {"ler_bp_only": k / shots, "ler_ci95": evaluate.wilson(k, shots),
                "osd_invoke_rate": float((r.converged == 0).float().mean().item()),
                "mean_iters": float(r.iters.float().mean().item())}

    out = {"workload": "rotated_d9_st9_p0.005", "shots": shots, "plain_bp": one(lottery=0), "policies": {}}
    for pol, name in names.items():
        out["policies"][name] = one(lottery=1, lottery_skip=6, lottery_policy=pol)
    out["skip_sweep_proposed"] = {str(s): one(lottery=1, lottery_skip=s, lottery_policy=0)
                                  for s in (0, 2, 4, 6, 8, 12)}
    dec.close()
    return out


def run_sum_product(shots: int = 1 << 17, seed: int = 43):
    """Check-node rule comparison: normalised min-sum (Alg. 1) against the
    sum-product tanh rule, with and without the lottery, on the rotated d=9
    surface code with 9 noisy rounds at p = 0.005 (BP alone: unconverged
    shots count as failures), then Lottery BP + OSD-0 throughput of each rule
    on the d=11 space-time workload (2^18 shots, tuned launch shape)."""
    import torch
    from paper_2605_00038_gb300 import evaluate, lbp
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler, workloads
    from paper_2605_00038_gb300.inputs.codes import rotated_surface, spacetime, spacetime_priors

    d, p = 9, 0.005
    hz, _ = rotated_surface(d)
    h = spacetime(hz, d)
    pri = spacetime_priors(hz, d, p, p)
    e, syn = sampler.sample(h, pri, seed=seed, num_shots=shots)
    spec = evaluate.surface_spec(d, d, h.n)
    true_d = torch.from_numpy(e.view(np.int64)).cuda()
    sd = torch.from_numpy(syn.view(np.int64)).cuda()
    dec = Decoder(h, pri)

    def one(**kw):
        r = dec.decode(sd, dec.params(max_iter=100, osd=0, seed=seed, **kw))
        torch.cuda.synchronize()
        f = evaluate.logical_failures(spec, true_d, r.err, r.converged, r.osd)
        k = int(f.sum().item())
        return {"ler_bp_only": k / shots, "ler_ci95": evaluate.wilson(k, shots),
                "osd_invoke_rate": float((r.converged == 0).float().mean().item()),
                "mean_iters": float(r.iters.float().mean().item())}

    MS, SPR = lbp.LBP_RULE_MIN_SUM, lbp.LBP_RULE_SUM_PRODUCT
    out = {"workload": "rotated_d9_st9_p0.005", "shots": shots, "quality": {
        "min_sum_plain_f32": one(rule=MS, lottery=0, msg=0),
        "min_sum_lottery_f32": one(rule=MS, lottery=1, msg=0),
        "sum_product_plain_f32": one(rule=SPR, lottery=0, msg=0),
        "sum_product_lottery_f32": one(rule=SPR, lottery=1, msg=0),
        "sum_product_lottery_f16": one(rule=SPR, lottery=1, msg=1)}}
    dec.close()

    w = workloads.c2_d11_spacetime(shots=1 << 18)
    _, syn2 = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=w.shots)
    x = torch.from_numpy(syn2.view(np.int64)).cuda()
    dec = Decoder(w.h, w.priors)
    thr = {}
    for name, rule, msg in (("min_sum_f32", MS, 0), ("sum_product_f32", SPR, 0),
                            ("sum_product_f16", SPR, 1)):
        prm = dec.params(**dict(w.decoder, rule=rule, msg=msg))
        dec.tune(x, prm)
        o = dec.alloc(w.shots)
        ws = dec.workspace(prm, w.shots)
        ms = []
        for r in range(4):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            lbp.lbp_decode(dec.code, prm, w.shots, x, o.err, o.converged, o.osd, o.iters, None, ws,
                           torch.cuda.current_stream().cuda_stream)
            b.record()
            b.synchronize()
            if r:
                ms.append(a.elapsed_time(b))
        thr[name] = {"shots_per_s": w.shots / (min(ms) / 1e3),
                     "osd_invoke_rate": float((o.converged == 0).float().mean().item())}
    dec.close()
    out["throughput_d11_st11_lottery_osd"] = thr
    return out


def main():
    args = parse()
    if args.serving_only:
        import __graft_entry__
        __graft_entry__.build()
        print(json.dumps({"serving": run_serving(), "matched_ler": run_matched(),
                          "precision": run_precision(), "lottery_design_space": run_policies(),
                          "check_rule": run_sum_product()}),
              flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
