#!/usr/bin/env python3
"""Throughput benchmark of the Lottery BP decoder on GB300.

One step = one pass of the whole decoding path (BP with the lottery on every
shot, early termination, hard decisions; this workload runs without OSD, as
configured) over one batch of seeded synthetic syndromes of the rotated d=25
surface code with 25 noisy rounds (space-time H 7,800 x 23,113, nnz 44,976),
p_data = p_meas = 0.004, max 100 iterations, binary32 messages.  A step
decodes 2^18 shots; four rotating batches of 2^18 make up the 2^20 shots of
the configuration (each 258 MB of syndromes, larger than L2).

Prints one JSON line (rank 0).  `value` is decoded shots per second over all
ranks with inputs resident in HBM; `e2e` is the same through the host-buffer
entry point with the copies inside the timed region.  Further legs (rank 0,
N = 1): the precision sweep of this workload (FP16 / INT8 messages, logical
error rates against the FP64 oracle), the rotated d=11 space-time workload
with Lottery BP + OSD-0, the BB [[144,12,12]] code with FP16 messages and
OSD-0, serving, matched LER, the lottery design space and the check-node
rule.  `--impl reference` times the CPU oracle instead (on a bounded sample
of the same workload).  Under torchrun each rank decodes its own shots (weak
scaling; no data-path collective).
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
N_BATCHES = 4        # rotating input batches of 2^18 shots: 4 x 258 MB of syndromes, each > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", choices=["d25", "d11", "bb144"], default="d25",
                    help="d25: the rotated d=25 space-time code, Lottery BP, FP32 (the headline); "
                         "d11: the rotated d=11 space-time code, Lottery BP + OSD-0, FP32; "
                         "bb144: BB [[144,12,12]] at p = 0.05, Lottery BP + OSD-0, FP16")
    ap.add_argument("--shots", type=int, default=None,
                    help="shots per step per rank (default 2^18 for d25, 10^6 for d11 and bb144)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip latency sweep, LER and CPU baseline")
    ap.add_argument("--cpu-sample", type=int, default=6144, help="oracle shots for cpu_baseline")
    ap.add_argument("--ref-sample", type=int, default=192, help="oracle shots per step of --impl reference")
    ap.add_argument("--no-tune", action="store_true", help="skip lbp_tune (default launch shape)")
    ap.add_argument("--rule", choices=["min_sum", "sum_product"], default="min_sum",
                    help="check-node rule of the main line (the configurations use min-sum)")
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


def workload(shots, which: str = "d25"):
    from paper_2605_00038_gb300.inputs import workloads
    if which == "d11":
        return workloads.c2_d11_spacetime(shots=shots or 1_000_000, osd=1)
    if which == "bb144":
        return workloads.c3_bb144(0.05, shots=shots or 1_000_000)
    return workloads.c5_d25_spacetime(msg=0, shots=shots or (1 << 18))


MSG_NAME = {0: "f32", 1: "f16", 2: "i8"}
MSG_BYTES = {0: 4, 1: 2, 2: 1}


def code_text(w):
    if w.name.startswith("bb144"):
        return "BB [[144,12,12]] H_X %dx%d nnz %d, code capacity" % (w.h.m, w.h.n, w.h.nnz)
    d = 25 if w.h.m == 7800 else 11
    return "rotated surface d=%d, %d noisy rounds, space-time H %dx%d nnz %d" % (d, d, w.h.m, w.h.n, w.h.nnz)


def state_bytes_per_iteration(h, msg_bytes):
    """Algorithmic bytes of one shot-iteration: the state that persists between
    iterations, read and written once: E messages of msg_bytes and n binary32
    posteriors, B_it = 2 (E b + 4 n)."""
    return 2 * (h.nnz * msg_bytes + 4 * h.n)


def io_bytes_per_shot(h):
    """Per shot: syndrome in, estimate out (packed 64-bit words), the
    converged flag, the OSD status byte and the iteration count."""
    return 8 * ((h.m + 63) // 64) + 8 * ((h.n + 63) // 64) + 1 + 1 + 4


def roofline_model(w, iters_total, shots):
    """Algorithmic work of K_bp: per shot-iteration 8 E + 2 m + n operations
    (per edge the V2C subtract, two minimum compares, sign parity, output
    select and sign, LLR add and syndrome XOR; per check two scale multiplies;
    per column the hard decision); per shot the syndrome in and results out."""
    E, m, n = w.h.nnz, w.h.m, w.h.n
    ops = float(iters_total) * (8 * E + 2 * m + n)
    io = shots * io_bytes_per_shot(w.h)
    return ops, io


# DRAM bytes of K_bp per shot-iteration on the d=25 workload (FP32 messages):
# dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of a
# 4,096-shot launch, divided by the shot-iterations it ran; the traffic of a
# full launch scales with its shot-iterations.  Valid for the kernel sources
# whose hash is recorded with it (None until captured).
KBP_TRAFFIC = {"bytes_per_shot_iteration": 12.30, "source_sha1": "e101fdb95106"}


def kbp_source_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in ("bp_ell_kernel.cuh", "bp_common.cuh", "bp_graph.cuh", "bp_lottery.cuh"):
        h.update((ROOT / "paper_2605_00038_gb300" / "csrc" / f).read_bytes())
    return h.hexdigest()[:12]


def alu_peak_ops(sm_mhz):
    # 152 SMs x 4 sub-partitions x 32 lanes, one instruction per lane per clock.
    return 152 * 4 * 32 * sm_mhz * 1e6


def hbm_peak_gbs():
    """(peak GB/s, basis): the measured copy bandwidth of the GB300s
    when MEASURED_PEAKS.json is present, else the recipe's fallback."""
    f = ROOT / "MEASURED_PEAKS.json"
    try:
        v = float(json.loads(f.read_text())["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def smem_bytes_per_iteration(h, msg_bytes):
    """On-chip bytes one shot-iteration must move: per edge the posterior and
    message read, the message written (check phase) and read again (column
    phase), E (4 + 3 b); per column the posterior written and the prior read,
    8 n."""
    return h.nnz * (4 + 3 * msg_bytes) + 8 * h.n


def smem_peak(stream=None, reps: int = 3):
    """(bytes/s, clock summary) of the shared-memory load bandwidth probe
    (lbp_probe_smem), the best of `reps` timed launches, with the SM clock
    sampled while it ran."""
    from paper_2605_00038_gb300 import lbp
    import torch
    cs = ClockSampler(torch.cuda.current_device())
    cs.start()
    best = 0.0
    t_end = time.perf_counter() + 0.5
    while True:
        for _ in range(reps):
            b, ms = lbp.lbp_probe_smem(4096, stream)
            best = max(best, b / (ms / 1e3))
        if time.perf_counter() >= t_end:
            break
    cs.stop()
    return best, cs.summary()


def histogram(iters_tensors):
    """Iteration histogram (Fig. 6) over the given per-shot iteration counts:
    {iterations: shots}, non-zero entries only."""
    import torch
    tot = None
    for t in iters_tensors:
        c = torch.bincount(t.to(torch.int64))
        if tot is None:
            tot = c
        else:
            if c.numel() > tot.numel():
                c, tot = tot, c
            tot[: c.numel()] += c
    nz = torch.nonzero(tot).flatten().tolist()
    vals = tot[nz].tolist()
    return {str(k): int(v) for k, v in zip(nz, vals)}


# ------------------------------------------------------------- reference arm

def oracle_params_for(w, oracle, prec=None):
    d = w.decoder
    return oracle.OracleParams(max_iter=d["max_iter"], scale_mode=d.get("scale_mode", 1),
                               scale_const=d.get("scale_const", 0.625), lottery=bool(d.get("lottery", 1)),
                               lottery_skip=d.get("lottery_skip", 6), osd=bool(d.get("osd", 0)),
                               prec=oracle.PREC_F64 if prec is None else prec, seed=w.seed)


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    from paper_2605_00038_gb300.inputs import sampler
    w = workload(args.shots, args.workload)
    cores = os.cpu_count() or 1
    sample = max(1, min(args.ref_sample, w.shots))
    _, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=sample * (args.steps + 1))
    S = sampler.unpack(syn, w.h.m)
    prm = oracle_params_for(w, oracle)
    for _ in range(args.warmup):
        oracle.decode(w.h, w.priors, S[: max(1, sample // 8)], prm, nthreads=cores)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.decode(w.h, w.priors, S[k * sample:(k + 1) * sample], prm, nthreads=cores)
    dt = time.perf_counter() - t0
    v = sample * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "shots_per_step": sample, "decoder": "lottery_bp",
                   "max_iter": w.decoder["max_iter"], "parallelism": "cpu threads"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d distinct shots of %s per step (FP64 oracle, %d threads)"
                                   % (sample, w.name, cores)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

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
    from paper_2605_00038_gb300 import evaluate, lbp
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler

    w = workload(args.shots, args.workload)
    if args.rule == "sum_product":
        w.decoder["rule"] = lbp.LBP_RULE_SUM_PRODUCT
    B = w.shots
    d25 = args.workload == "d25"
    msg = w.decoder["msg"]
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
        o = outs[k % N_BATCHES]
        lbp.lbp_decode(dec.code, prms[k % N_BATCHES], B, syn_d[k % N_BATCHES], o.err, o.converged, o.osd,
                       o.iters, None, ws, stream)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # Launch-shape autotuning on part of the first batch (outside the timed region).
    launch = None
    if not args.no_tune:
        tb = min(B, 16384)
        dec.tune(syn_d[0][:tb].contiguous(), prms[0], stream)
        S_t, G_t, gf_t = lbp.lbp_code_tuned(dec.code, prms[0].msg, prms[0].rule)
        launch = {"groups_per_cta": S_t, "threads_per_shot": G_t,
                  "graph": {0: "default", 1: "index image", 2: "implicit", 3: "round"}.get(gf_t, str(gf_t))}
        _, S_e, G_e, _, _ = lbp.lbp_code_options(dec.code)
        if S_e and G_e:          # LBP_BP_SHAPE, read at load, takes precedence over the tuned shape
            launch.update(groups_per_cta=S_e, threads_per_shot=G_e, source="LBP_BP_SHAPE")
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

    # Work actually done in the timed steps (iterations per batch decoded).
    iters_total = 0
    unconverged = 0
    osd_total = 0
    for k in range(args.steps):
        o = outs[k % N_BATCHES]
        iters_total += int(o.iters.sum().item())
        unconverged += int((o.converged == 0).sum().item())
        osd_total += int((o.osd != 0).sum().item())
    hist = histogram([outs[k].iters for k in range(min(args.steps, N_BATCHES))])

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": MSG_NAME[msg], "data": "synthetic",
        "config": {"workload": w.name, "code": code_text(w),
                   "noise": {"d25": "iid p_data=p_meas=0.004", "d11": "iid p_data=p_meas=0.003",
                             "bb144": "iid p=0.05"}[args.workload],
                   "shots_per_step_per_rank": B, "configuration_shots": N_BATCHES * B,
                   "decoder": "lottery_bp(proposed rule, skip 6, adaptive scale, I=100)" +
                              (", no OSD" if d25 else " + osd0"),
                   "msg": MSG_NAME[msg], "check_rule": args.rule,
                   "l2": "%d rotating input batches of %d MB syndromes, each > L2" % (
                       N_BATCHES, B * wm * 8 // 2 ** 20),
                   "parallelism": "replicas" if world > 1 else "single"},
        "clocks": clocks.summary(),
        "gpu_launches": int(bp_n + osd_n),
    }
    sm_mhz = line["clocks"]["sm_mhz"] or 2070.0
    iters_per_step = iters_total / args.steps
    bp_avg_s = bp_ms / max(bp_n, 1) / 1e3
    b_it = state_bytes_per_iteration(w.h, MSG_BYTES[msg])
    alg_bytes = iters_per_step * b_it + B * io_bytes_per_shot(w.h)
    peak_gbs, peak_basis = hbm_peak_gbs()
    traffic = None
    if d25 and KBP_TRAFFIC["bytes_per_shot_iteration"] and kbp_source_sha1() == KBP_TRAFFIC["source_sha1"]:
        traffic = KBP_TRAFFIC["bytes_per_shot_iteration"] * iters_per_step
    ops, _ = roofline_model(w, iters_per_step, B)
    line["roofline"] = {
        "bound": "hbm", "achieved": alg_bytes / bp_avg_s / 1e9, "peak": peak_gbs, "unit": "GB/s",
        "frac": alg_bytes / bp_avg_s / 1e9 / peak_gbs, "traffic": traffic,
        "kernel": "bp_ell_kernel", "avg_launch_ms": bp_avg_s * 1e3,
        "bytes_per_shot_iteration": b_it, "shot_iterations_per_launch": iters_per_step,
        "algorithmic_bytes_per_launch": alg_bytes, "peak_basis": peak_basis,
        "dram_gbs_from_traffic": (traffic / bp_avg_s / 1e9) if traffic else None,
        "note": "algorithmic bytes = state read and written once per shot-iteration, 2 (E b + 4 n), "
                "plus I/O" + ("; the posteriors, syndrome words and four of six message slots stay in "
                              "shared memory, the other two slots in an L2-resident workspace slice, so "
                              "DRAM carries far less than the algorithmic bytes (traffic)" if d25 else
                              "; the whole state stays in shared memory"),
        "alu": {"achieved_tops": ops / bp_avg_s / 1e12, "peak_tops": alu_peak_ops(sm_mhz) / 1e12,
                "frac": ops / bp_avg_s / alu_peak_ops(sm_mhz),
                "peak_basis": "152 SMs x 128 lanes x median SM clock %.0f MHz (derived)" % sm_mhz}}
    smem_bps, smem_clk = smem_peak(stream)
    smem_alg = iters_per_step * smem_bytes_per_iteration(w.h, MSG_BYTES[msg])
    line["roofline"]["smem"] = {"achieved_tbs": smem_alg / bp_avg_s / 1e12, "peak_tbs": smem_bps / 1e12,
                                "frac": smem_alg / bp_avg_s / smem_bps,
                                "bytes_per_shot_iteration": smem_bytes_per_iteration(w.h, MSG_BYTES[msg]),
                                "peak_basis": "measured by lbp_probe_smem (conflict-free 16-byte loads), "
                                              "SM clock %s MHz while it ran" % smem_clk.get("sm_mhz")}
    line["kernels"] = {"bp_launch": launch, "bp_ms_per_step": bp_ms / args.steps,
                       "osd_ms_per_step": osd_ms / args.steps,
                       "mean_iters": iters_total / (B * args.steps),
                       "unconverged_rate": unconverged / (B * args.steps),
                       "osd_invoke_rate": osd_total / (B * args.steps),
                       "iteration_histogram": hist}

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
        # Per-batch latency (outside the timed region): each repeat decodes
        # different shots of batch 0.
        line["latency"] = latency_sweep(dec, prms[0], syn_d[0], ((1, 30), (64, 12), (4096, 5)), stream)
        line["latency"]["batch_%d" % B] = {"p50_ms": line["ms_per_step"], "p99_ms": None}
        # Logical error rate of batch 0 (true errors known from the sampler).
        o = outs[0]
        step(0)
        torch.cuda.synchronize()
        spec = {"d25": lambda: evaluate.surface_spec(25, 25, w.h.n),
                "d11": lambda: evaluate.surface_spec(11, 11, w.h.n),
                "bb144": lambda: evaluate.bb_spec("bb144")}[args.workload]()
        f = evaluate.logical_failures(spec, torch.from_numpy(err_h[0].view(np.int64)).cuda(), o.err,
                                      o.converged, o.osd)
        k = int(f.sum().item())
        line["quality"] = {"ler": k / B, "ler_ci95": evaluate.wilson(k, B), "shots": B, "logical_failures": k,
                           "note": "BP alone (no OSD in this configuration): an unconverged shot counts as a "
                                   "logical failure" if d25 else "Lottery BP + OSD-0"}

    if not args.no_extras and rank == 0 and world == 1 and d25:
        del outs, ws
        dec.close()
        torch.cuda.empty_cache()
        line["precision_d25"] = run_c5_precision(syn_h[0], err_h[0], args)
        line["d11_spacetime_osd"] = run_c2_leg(args)
        line["bb144_osd_fp16"] = run_c3_leg()
        line["serving"] = run_serving()
        line["serving_one_launch_fifo"] = run_serving(policy=(0, False))
        line["serving_merged"] = run_serving(merge=16)
        line["matched_ler"] = run_matched()
        line["precision_d7"] = run_precision()
        line["lottery_design_space"] = run_policies()
        line["check_rule"] = run_sum_product()
    else:
        dec.close()
    if not args.no_extras and rank == 0 and world == 1 and d25:
        import oracle
        cores = os.cpu_count() or 1
        S = sampler.unpack(syn_h[0][: args.cpu_sample], w.h.m)
        t0 = time.perf_counter()
        oracle.decode(w.h, w.priors, S, oracle_params_for(w, oracle), nthreads=cores)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": S.shape[0] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%d shots of %s (FP64 oracle, %d threads, %.1f s)"
                                          % (S.shape[0], w.name, cores, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def latency_sweep(dec, prm, syn_d, sizes, stream):
    """Per-batch latency quantiles (CUDA events around lbp_decode), each repeat
    on different shots of syn_d; the first two repeats are warm-up."""
    import torch
    from paper_2605_00038_gb300 import lbp
    lat = {}
    B = syn_d.shape[0]
    for bs, reps in sizes:
        o = dec.alloc(bs)
        wsb = dec.workspace(prm, bs)
        times = []
        for r in range(reps + 2):
            lo = (r * bs) % max(1, B - bs + 1)
            sub = syn_d[lo:lo + bs].contiguous()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lbp.lbp_decode(dec.code, prm, bs, sub, o.err, o.converged, o.osd, o.iters, None, wsb, stream)
            b.record(stream)
            b.synchronize()
            if r >= 2:
                times.append(a.elapsed_time(b))
        times.sort()
        lat["batch_%d" % bs] = {"p50_ms": times[len(times) // 2],
                                "p99_ms": times[min(len(times) - 1, int(0.99 * len(times)))],
                                "samples": len(times)}
    return lat


def run_c5_precision(syn0, err0, args, timed_shots: int = 1 << 18, oracle_shots: int = 4096):
    """Precision sweep of the d=25 workload (rotated d=25 space-time code, 2^20 shots):
    FP32 / FP16 / INT8 messages on the same shots, each timed on one batch of
    2^18 shots (tuned launch shape), with its logical error rate (BP alone, an
    unconverged shot fails) and the paired comparison with the FP64 oracle on
    the first `oracle_shots` shots.  Then the same decoder on the unrotated
    d=25 space-time code (Table III, 15,000 x 44,425) at the same noise, where
    BP converges far more often: the rotated code's weight-2 boundary checks
    make degenerate pairs that stall BP (shown at d=11 too)."""
    import torch
    import oracle
    from paper_2605_00038_gb300 import evaluate
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler, workloads
    from paper_2605_00038_gb300.inputs.codes import spacetime, spacetime_priors, unrotated_surface

    w = workloads.c5_d25_spacetime(msg=0, shots=timed_shots)
    spec = evaluate.surface_spec(25, 25, w.h.n)
    x = torch.from_numpy(syn0[:timed_shots].view(np.int64)).cuda()
    true_d = torch.from_numpy(err0[:timed_shots].view(np.int64)).cuda()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.decode(w.h, w.priors, sampler.unpack(syn0[:oracle_shots], w.h.m),
                      oracle_params_for(w, oracle), nthreads=cores)
    t_or = time.perf_counter() - t0
    fo = evaluate.logical_failures(spec, true_d[:oracle_shots].cpu(),
                                   torch.from_numpy(sampler.pack(r.err).view(np.int64)),
                                   torch.from_numpy(r.converged), torch.from_numpy(r.osd_used)).numpy()
    ko = int(fo.sum())
    out = {"workload": w.name, "timed_shots": timed_shots, "oracle_shots": oracle_shots,
           "fp64_oracle": {"ler": ko / oracle_shots, "ler_ci95": evaluate.wilson(ko, oracle_shots),
                           "unconverged_rate": float(1.0 - r.converged.mean()),
                           "seconds": t_or, "threads": cores}}
    dec = Decoder(w.h, w.priors)
    for msg, name in ((0, "fp32"), (1, "fp16"), (2, "int8")):
        prm = dec.params(**dict(w.decoder, msg=msg), seed=w.seed)
        dec.tune(x[:16384].contiguous(), prm)
        dec.decode(x[:4096].contiguous(), prm)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        res = dec.decode(x, prm)
        a1.record()
        torch.cuda.synchronize()
        t = a0.elapsed_time(a1) / 1e3
        it = float(res.iters.float().mean().item())
        f = evaluate.logical_failures(spec, true_d, res.err, res.converged, res.osd).cpu().numpy()
        k = int(f.sum())
        fs = f[:oracle_shots]
        S_t, G_t, gf_t = lbp_tuned(dec, prm)
        out[name] = {"shots_per_s": timed_shots / t, "mean_iters": it,
                     "unconverged_rate": float((res.converged == 0).float().mean().item()),
                     "state_bytes_per_shot_iteration": state_bytes_per_iteration(w.h, {0: 4, 1: 2, 2: 1}[msg]),
                     "launch": {"groups_per_cta": S_t, "threads_per_shot": G_t, "graph": gf_t},
                     "ler": k / timed_shots, "ler_ci95": evaluate.wilson(k, timed_shots),
                     "ler_subset": float(fs.mean()), "gap_vs_fp64_subset": float(fs.mean() - fo.mean()),
                     "mcnemar_p_vs_fp64": evaluate.mcnemar_p(int((fs & ~fo).sum()), int((fo & ~fs).sum()))}
    dec.close()
    # The paper's own family (Table III): unrotated d=25, 25 rounds, same noise.
    _, hz = unrotated_surface(25)
    st = spacetime(hz, 25)
    pri = spacetime_priors(hz, 25, 0.004, 0.004)
    n_u = 1 << 14
    _, su = sampler.sample(st, pri, seed=w.seed, num_shots=n_u)
    xu = torch.from_numpy(su.view(np.int64)).cuda()
    du = Decoder(st, pri)
    unrot = {"shape": [st.m, st.n, st.nnz], "shots": n_u}
    for I in (100, 300):
        for lot in (0, 1):
            prm = du.params(max_iter=I, lottery=lot, osd=0, msg=0, seed=w.seed)
            res = du.decode(xu, prm)
            torch.cuda.synchronize()
            unrot["%s_I%d" % ("lottery" if lot else "plain", I)] = {
                "unconverged_rate": float((res.converged == 0).float().mean().item()),
                "mean_iters": float(res.iters.float().mean().item())}
    du.close()
    out["unrotated_d25_st25_p0.004"] = unrot
    return out


def lbp_tuned(dec, prm):
    from paper_2605_00038_gb300 import lbp
    return lbp.lbp_code_tuned(dec.code, prm.msg, prm.rule)


def run_c2_leg(args, shots: int = 1_000_000, steps: int = 5, warmup: int = 3):
    """The rotated d=11 space-time workload (10^6 shots, Lottery BP + OSD-0, FP32):
    Lottery BP + OSD-0, FP32 messages, 10^6 shots per step, three rotating
    batches (88 MB of syndromes each), tuned launch shape; shots/s device
    resident and end to end, kernel times, OSD invoke rate, iteration
    histogram, small-batch latency, logical error rate."""
    import torch
    from paper_2605_00038_gb300 import evaluate, lbp
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler, workloads

    w = workloads.c2_d11_spacetime(shots=shots, osd=1)
    B = w.shots
    nb = 3
    dec = Decoder(w.h, w.priors)
    wm, wn = (w.h.m + 63) // 64, (w.h.n + 63) // 64
    syn_h, err_h, syn_d, prms = [], [], [], []
    for k in range(nb):
        e, s = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=B, shot_offset=k * B)
        err_h.append(e)
        syn_h.append(s)
        syn_d.append(torch.from_numpy(s.view(np.int64)).cuda())
        prms.append(dec.params(**w.decoder, seed=w.seed, shot_offset=k * B))
    outs = [dec.alloc(B) for _ in range(nb)]
    ws = dec.workspace(prms[0], B)
    stream = torch.cuda.current_stream()
    dec.tune(syn_d[0][:131072].contiguous(), prms[0], stream)

    def step(k):
        o = outs[k % nb]
        lbp.lbp_decode(dec.code, prms[k % nb], B, syn_d[k % nb], o.err, o.converged, o.osd, o.iters, None, ws,
                       stream)

    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()
    lbp.lbp_timing_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        step(k)
    e1.record(stream)
    torch.cuda.synchronize()
    bp_ms, bp_n, osd_ms, osd_n = lbp.lbp_timing_read()
    lbp.lbp_timing_enable(False)
    t = e0.elapsed_time(e1) / 1e3
    iters = sum(int(outs[k % nb].iters.sum().item()) for k in range(steps))
    osd_total = sum(int((outs[k % nb].osd != 0).sum().item()) for k in range(steps))
    S_t, G_t, gf_t = lbp_tuned(dec, prms[0])
    out = {"workload": w.name, "shots_per_step": B, "steps": steps, "shots_per_s": B * steps / t,
           "ms_per_step": 1e3 * t / steps, "bp_ms_per_step": bp_ms / steps, "osd_ms_per_step": osd_ms / steps,
           "bp_launch": {"groups_per_cta": S_t, "threads_per_shot": G_t, "graph": gf_t},
           "mean_iters": iters / (B * steps), "osd_invoke_rate": osd_total / (B * steps),
           "iteration_histogram": histogram([outs[k].iters for k in range(nb)])}
    # ALU and shared-memory views of K_bp (the state stays in shared memory).
    ops, _ = roofline_model(w, iters / steps, B)
    bp_avg_s = bp_ms / max(bp_n, 1) / 1e3
    smem_bps, _ = smem_peak()
    out["roofline_alu"] = {"achieved_tops": ops / bp_avg_s / 1e12, "frac": ops / bp_avg_s / alu_peak_ops(2070.0),
                           "algorithmic_state_tbs": (iters / steps) * state_bytes_per_iteration(w.h, 4)
                                                    / bp_avg_s / 1e12}
    out["roofline_smem"] = {"achieved_tbs": (iters / steps) * smem_bytes_per_iteration(w.h, 4) / bp_avg_s / 1e12,
                            "peak_tbs": smem_bps / 1e12,
                            "frac": (iters / steps) * smem_bytes_per_iteration(w.h, 4) / bp_avg_s / smem_bps}
    # End to end through the host-buffer entry point.
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()
    hsyn = pin(syn_h[0].shape, torch.int64)
    hsyn.numpy()[:] = syn_h[0].view(np.int64)
    ho = dict(err=pin((B, wn), torch.int64), converged=pin(B, torch.uint8), osd=pin(B, torch.uint8),
              iters=pin(B, torch.int32))
    hws = dec.workspace(prms[0], B, host=True)
    lbp.lbp_decode_host(dec.code, prms[0], B, hsyn, ho["err"], ho["converged"], ho["osd"], ho["iters"], None,
                        hws, stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for k in range(steps):
        lbp.lbp_decode_host(dec.code, prms[0], B, hsyn, ho["err"], ho["converged"], ho["osd"], ho["iters"],
                            None, hws, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    out["e2e_shots_per_s"] = B * steps / (e0.elapsed_time(e1) / 1e3)
    # Small-batch latency, each repeat on different shots; batch 1 replayed
    # from a CUDA graph too.
    out["latency"] = latency_sweep(dec, prms[0], syn_d[0], ((1, 200), (64, 200), (4096, 50)), stream)
    x1 = torch.empty((1, wm), dtype=torch.int64, device="cuda")
    o1 = dec.alloc(1)
    ws1 = torch.empty(lbp.lbp_workspace_size(dec.code, prms[0], 1) + 256, dtype=torch.uint8, device="cuda")
    ws1 = ws1[(-ws1.data_ptr()) % 256:]
    g1 = lbp.lbp_graph_create(dec.code, prms[0], 1, x1, o1.err, o1.converged, o1.osd, o1.iters, None, ws1)
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
    out["latency"]["batch_1_graph"] = {"p50_ms": times[len(times) // 2],
                                       "p99_ms": times[min(len(times) - 1, int(0.99 * len(times)))],
                                       "samples": len(times)}
    step(0)
    torch.cuda.synchronize()
    o = outs[0]
    f = evaluate.logical_failures(evaluate.surface_spec(11, 11, w.h.n),
                                  torch.from_numpy(err_h[0].view(np.int64)).cuda(), o.err, o.converged, o.osd)
    k = int(f.sum().item())
    out["ler"] = k / B
    out["ler_ci95"] = evaluate.wilson(k, B)
    dec.close()
    return out


def run_c3_leg(shots: int = 1_000_000, oracle_shots: int = 100_000):
    """BB [[144,12,12]] code capacity (10^6 shots per p, Lottery BP + OSD-0, FP16):
    Lottery BP + OSD-0 with FP16 messages, p in {0.01, 0.03, 0.05}, 10^6 shots
    each (tuned launch shape): shots/s, OSD invoke rate, mean iterations,
    logical error rate with its Wilson interval, and the paired comparison
    with the FP64 oracle on the first `oracle_shots` shots."""
    import torch
    import oracle
    from paper_2605_00038_gb300 import evaluate
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler, workloads

    spec = evaluate.bb_spec("bb144")
    cores = os.cpu_count() or 1
    out = {}
    for p in (0.01, 0.03, 0.05):
        w = workloads.c3_bb144(p, shots=shots)
        e, syn = sampler.sample(w.h, w.priors, seed=w.seed, num_shots=shots)
        x = torch.from_numpy(syn.view(np.int64)).cuda()
        true_d = torch.from_numpy(e.view(np.int64)).cuda()
        dec = Decoder(w.h, w.priors)
        prm = dec.params(**w.decoder, seed=w.seed)
        dec.tune(x[:131072].contiguous(), prm)
        dec.decode(x, prm)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        res = dec.decode(x, prm)
        a1.record()
        torch.cuda.synchronize()
        t = a0.elapsed_time(a1) / 1e3
        f = evaluate.logical_failures(spec, true_d, res.err, res.converged, res.osd).cpu().numpy()
        k = int(f.sum())
        t0 = time.perf_counter()
        r = oracle.decode(w.h, w.priors, sampler.unpack(syn[:oracle_shots], w.h.m), oracle_params_for(w, oracle),
                          nthreads=cores)
        t_or = time.perf_counter() - t0
        fo = evaluate.logical_failures(spec, true_d[:oracle_shots].cpu(),
                                       torch.from_numpy(sampler.pack(r.err).view(np.int64)),
                                       torch.from_numpy(r.converged), torch.from_numpy(r.osd_used)).numpy()
        fs = f[:oracle_shots]
        S_t, G_t, gf_t = lbp_tuned(dec, prm)
        out["p%g" % p] = {
            "workload": w.name, "shots": shots, "shots_per_s": shots / t,
            "launch": {"groups_per_cta": S_t, "threads_per_shot": G_t, "graph": gf_t},
            "osd_invoke_rate": float((res.osd != 0).float().mean().item()),
            "mean_iters": float(res.iters.float().mean().item()),
            "ler": k / shots, "ler_ci95": evaluate.wilson(k, shots),
            "fp64_oracle_subset": {"shots": oracle_shots, "ler": float(fo.mean()),
                                   "shots_per_s": oracle_shots / t_or, "threads": cores},
            "gap_vs_fp64_subset": float(fs.mean() - fo.mean()),
            "mcnemar_p_vs_fp64": evaluate.mcnemar_p(int((fs & ~fo).sum()), int((fo & ~fs).sum()))}
        dec.close()
    return out


def run_serving(seconds_per_rate: float = 3.0, n_requests: int = 600, seed: int = 11, policy=None, merge: int = 0):
    """Serving mix: Poisson arrivals of 1-4096-shot requests over ten resident
    codes (rotated surface space-time d = 5..17 with d rounds, BB 72/144/288
    code capacity) and five noise levels 1e-3..5e-3; Lottery BP + OSD-0,
    I = 100, INT8 messages.  Capacity first (all requests queued at once), then
    open-loop arrivals at 50 / 80 / 95 % of it.  Messages are Int3.4 (INT8),
    the format the paper's hardware uses; FP16 messages roughly double the
    lottery's OSD invoke rate on these surface codes.  policy: None for the
    server's default scheduling (launches of at most 16 Mi edge-shots,
    single-launch requests on a high-priority stream), or (chunk_work,
    priority) for lbp_server_configure; merge > 0 lets the server put up to
    that many compatible requests into one BP launch (lbp_server_set_batching)."""
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
    if merge:
        lbp.lbp_server_set_batching(srv, merge)

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
    # The same shots decoded as large device-resident batches, one per code and
    # noise level (8,192 shots each, default launch shape): the time the mix's
    # shots would take without serving (no copies, no small launches).
    rate = {}
    for key, dec in decs.items():
        used = [r for r in reqs if (r["ci"], r["pi"]) == key]
        if not used:
            continue
        h = dec.h
        nb = 8192
        _, sb = sampler.sample(h, dec_priors(dec), seed=seed + 1000 + key[0], num_shots=nb)
        x = torch.from_numpy(sb.view(np.int64)).cuda()
        prm = dec.params(max_iter=100, lottery=1, osd=1, msg=2, seed=seed)
        dec.decode(x, prm)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        dec.decode(x, prm)
        e1.record()
        torch.cuda.synchronize()
        rate[key] = nb / (e0.elapsed_time(e1) / 1e3)
    ideal_s = sum(r["B"] / rate[(r["ci"], r["pi"])] for r in reqs)
    out = {"policy": ("chunk_work 16 Mi edge-shots, priority" if policy is None else
                      "chunk_work %d, priority %d" % (policy[0], int(policy[1]))) +
                     (", merged launches of up to %d requests" % merge if merge else ""),
           "batched_equivalent_shots_per_s": total_shots / ideal_s,
           "serving_efficiency": (total_shots / dt) / (total_shots / ideal_s),
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


def _served(dec, prms, hs, hbuf, load, rng):
    """Serve the requests (lo, B, params) through one lbp_server: capacity with
    all queued, then open-loop Poisson arrivals at `load` x that capacity.
    Returns (capacity shots/s, open-loop dict, request latencies of the
    capacity run)."""
    import torch
    from paper_2605_00038_gb300 import lbp
    herr, hconv, hosd, hit = hbuf
    srv = lbp.lbp_server_create(8 << 30, 16)

    def submit(lo, B, prm):
        return lbp.lbp_server_submit(srv, dec.code, prm, B, hs[lo:lo + B], herr[lo:lo + B], hconv[lo:lo + B],
                                     hosd[lo:lo + B], hit[lo:lo + B])

    lo0, B0, p0 = prms[0]
    lbp.lbp_server_wait(srv, submit(lo0, B0, p0))
    total = sum(B for _, B, _ in prms)
    t0 = time.perf_counter()
    tks = [submit(lo, B, prm) for lo, B, prm in prms]
    for t in tks:
        lbp.lbp_server_wait(srv, t)
    span = time.perf_counter() - t0
    cap = total / span
    rate = load * len(prms) / span
    gaps = rng.exponential(1.0 / rate, size=len(prms))
    sent = []
    t_start = time.perf_counter()
    t_next = t_start
    for j, (lo, B, prm) in enumerate(prms):
        t_next += gaps[j]
        while True:
            now = time.perf_counter()
            if now >= t_next:
                break
            time.sleep(min(0.0005, t_next - now))
        sent.append(submit(lo, B, prm))
    lats = [lbp.lbp_server_wait(srv, t) for t in sent]
    span2 = time.perf_counter() - t_start
    srv.close()
    q = lambda x: float(np.quantile(np.asarray(lats), x) * 1e3)
    return cap, {"load": load, "offered_requests_per_s": rate, "requests": len(prms),
                 "shots_per_s": total / span2, "p50_ms": q(0.5), "p99_ms": q(0.99)}


def run_matched(shots: int = 1 << 20, request: int = 4096, seed: int = 21, load: float = 0.8):
    """Matched-LER head-to-head on identical shots: (A) plain NMS BP + OSD-0
    with FP32 messages against Lottery BP + OSD-0 with INT8 (Int3.4) messages
    and the paper's rule (Alg. 3), with the worst-check /
    least-reliable-column rule of Sec. III-B, and with Alg. 3 drawing from
    this iteration's s_hat instead of the previous one (an ablation of the
    delay the paper adopts for pipelining), on the code families the paper
    evaluates (the BB [[144,12,12]] code at p = 0.03 and 0.05, code capacity;
    the unrotated surface code's space-time matrix, Table III rows, d = 7,
    7 rounds, p = 0.01) and on the rotated d = 7 space-time code (p = 0.012);
    at BB144 p = 0.05 also the lottery's start iteration (6, 12, 20, 40).  Every
    arm is timed the same two ways: one device-resident lbp_decode of all
    shots, and served through lbp_server from host buffers in 4096-shot
    requests (capacity with every request queued; then open-loop Poisson
    arrivals at 80% of that arm's own capacity, whose p50 / p99 request
    latency is not queueing).  LER with Wilson intervals and the paired
    McNemar test of each Lottery arm against (A)."""
    import torch
    from paper_2605_00038_gb300 import evaluate, lbp
    from paper_2605_00038_gb300.decoder import Decoder
    from paper_2605_00038_gb300.inputs import sampler
    from paper_2605_00038_gb300.inputs.codes import (bb_code, rotated_surface, spacetime, spacetime_priors,
                                                     unrotated_surface)

    fams = []
    hx, _ = bb_code("bb144")
    fams.append(("bb144_cc_p0.03", hx, np.full(hx.n, 0.03), evaluate.bb_spec("bb144")))
    fams.append(("bb144_cc_p0.05", hx, np.full(hx.n, 0.05), evaluate.bb_spec("bb144")))
    _, uz = unrotated_surface(7)
    ust = spacetime(uz, 7)
    fams.append(("unrotated_d7_st7_p0.01", ust, spacetime_priors(uz, 7, 0.01, 0.01),
                 evaluate.unrotated_surface_spec(7, 7, ust.n)))
    rz, _ = rotated_surface(7)
    rst = spacetime(rz, 7)
    fams.append(("rotated_d7_st7_p0.012", rst, spacetime_priors(rz, 7, 0.012, 0.012),
                 evaluate.surface_spec(7, 7, rst.n)))
    rng = np.random.default_rng(seed)
    out = {"shots": shots, "request_shots": request, "open_loop_load": load, "families": {}}
    for name, h, pri, spec in fams:
        e, syn = sampler.sample(h, pri, seed=seed, num_shots=shots)
        true_d = torch.from_numpy(e.view(np.int64)).cuda()
        sd = torch.from_numpy(syn.view(np.int64)).cuda()
        dec = Decoder(h, pri)
        pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory()
        hs = pin(syn.shape, torch.int64)
        hs.numpy()[:] = syn.view(np.int64)
        wn = (h.n + 63) // 64
        hbuf = (pin((shots, wn), torch.int64), pin(shots, torch.uint8), pin(shots, torch.uint8),
                pin(shots, torch.int32))
        arms = [("plain_bp_osd_fp32", dict(lottery=0, msg=0, lottery_policy=0)),
                ("lottery_alg3_bp_osd_int8", dict(lottery=1, msg=2, lottery_policy=lbp.LBP_LOTTERY_PROPOSED)),
                ("lottery_worst_unreliable_bp_osd_int8",
                 dict(lottery=1, msg=2, lottery_policy=lbp.LBP_LOTTERY_WORST_UNRELIABLE)),
                # Alg. 3 with U from this iteration's s_hat (an ablation of its delay).
                ("lottery_alg3_current_syndrome_bp_osd_int8",
                 dict(lottery=1, msg=2, lottery_policy=lbp.LBP_LOTTERY_PROPOSED_CURRENT))]
        fam = {"shape": [h.m, h.n, h.nnz]}
        fa = None
        for arm, kw in arms:
            prm = dec.params(max_iter=100, osd=1, seed=seed, **kw)
            dec.decode(sd[:4096].contiguous(), prm)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            r = dec.decode(sd, prm)
            a1.record()
            torch.cuda.synchronize()
            tb = a0.elapsed_time(a1) / 1e3
            f = evaluate.logical_failures(spec, true_d, r.err, r.converged, r.osd)
            k = int(f.sum().item())
            reqs = [(lo, min(request, shots - lo), dec.params(max_iter=100, osd=1, seed=seed, shot_offset=lo, **kw))
                    for lo in range(0, shots, request)]
            cap, ol = _served(dec, reqs, hs, hbuf, load, rng)
            same = bool(torch.equal(hbuf[0].cuda(), r.err) and torch.equal(hbuf[1].cuda(), r.converged))
            res = {"ler": k / shots, "ler_ci95": evaluate.wilson(k, shots), "logical_failures": k,
                   "batched_shots_per_s": shots / tb, "served_capacity_shots_per_s": cap, "served_open_loop": ol,
                   "served_equals_batched": same,
                   "osd_invoke_rate": float((r.osd != 0).float().mean().item()),
                   "mean_iters": float(r.iters.float().mean().item())}
            if fa is None:
                fa, ka = f, k
            else:
                only_a = int((fa & ~f).sum().item())
                only_b = int((f & ~fa).sum().item())
                res.update({"ler_relative_difference": (k - ka) / max(ka, 1),
                            "mcnemar_discordant": [only_a, only_b],
                            "mcnemar_p": evaluate.mcnemar_p(only_a, only_b)})
            fam[arm] = res
        if name == "bb144_cc_p0.05":
            # The lottery's start iteration (Sec. III-B skips 6, chosen at low
            # p): Alg. 3 + OSD-0, INT8, batched, against the plain arm above.
            sweep = {}
            for skip in (6, 12, 20, 40):
                prm = dec.params(max_iter=100, osd=1, seed=seed, lottery=1, msg=2, lottery_skip=skip)
                r = dec.decode(sd, prm)
                torch.cuda.synchronize()
                f = evaluate.logical_failures(spec, true_d, r.err, r.converged, r.osd)
                k = int(f.sum().item())
                sweep[str(skip)] = {"ler": k / shots, "ler_relative_difference": (k - ka) / max(ka, 1),
                                    "osd_invoke_rate": float((r.osd != 0).float().mean().item()),
                                    "mean_iters": float(r.iters.float().mean().item())}
            fam["lottery_alg3_skip_sweep"] = sweep
        # The iteration cap: the same shots at I = 300 (the cap the paper's
        # accuracy comparisons quote), batched, each arm against plain BP +
        # OSD-0 at I = 100 above and at I = 300.
        cap = {}
        f300 = None
        for arm, kw in (("plain_bp_osd_fp32", dict(lottery=0, msg=0)),
                        ("lottery_alg3_bp_osd_int8", dict(lottery=1, msg=2)),
                        ("lottery_alg3_bp_osd_fp32", dict(lottery=1, msg=0)),
                        ("lottery_worst_unreliable_bp_osd_int8",
                         dict(lottery=1, msg=2, lottery_policy=lbp.LBP_LOTTERY_WORST_UNRELIABLE))):
            prm = dec.params(max_iter=300, osd=1, seed=seed, **kw)
            r = dec.decode(sd, prm)
            torch.cuda.synchronize()
            f = evaluate.logical_failures(spec, true_d, r.err, r.converged, r.osd)
            k = int(f.sum().item())
            res = {"ler": k / shots, "osd_invoke_rate": float((r.osd != 0).float().mean().item()),
                   "mean_iters": float(r.iters.float().mean().item()),
                   "ler_relative_difference_vs_plain_i100": (k - ka) / max(ka, 1),
                   "mcnemar_p_vs_plain_i100": evaluate.mcnemar_p(int((fa & ~f).sum().item()),
                                                                 int((f & ~fa).sum().item()))}
            if f300 is None:
                f300, k300 = f, k
            else:
                res["ler_relative_difference_vs_plain_i300"] = (k - k300) / max(k300, 1)
                res["mcnemar_p_vs_plain_i300"] = evaluate.mcnemar_p(int((f300 & ~f).sum().item()),
                                                                    int((f & ~f300).sum().item()))
            cap[arm] = res
        fam["iteration_cap_300"] = cap
        # Ablation of the lottery's delay (reading R6): Alg. 3 with U from this
        # iteration's s_hat (policy 5), INT8, batched, at I = 300 (its I = 100
        # arm is served above).
        abl = {}
        for cap_i, ref_f, ref_k in ((300, f300, k300),):
            prm = dec.params(max_iter=cap_i, osd=1, seed=seed, lottery=1, msg=2,
                             lottery_policy=lbp.LBP_LOTTERY_PROPOSED_CURRENT)
            r = dec.decode(sd, prm)
            torch.cuda.synchronize()
            f = evaluate.logical_failures(spec, true_d, r.err, r.converged, r.osd)
            k = int(f.sum().item())
            abl["I%d" % cap_i] = {"ler": k / shots, "osd_invoke_rate": float((r.osd != 0).float().mean().item()),
                                  "mean_iters": float(r.iters.float().mean().item()),
                                  "ler_relative_difference_vs_plain_same_cap": (k - ref_k) / max(ref_k, 1),
                                  "mcnemar_p_vs_plain_same_cap": evaluate.mcnemar_p(
                                      int((ref_f & ~f).sum().item()), int((f & ~ref_f).sum().item()))}
        fam["lottery_alg3_current_syndrome_int8"] = abl
        out["families"][name] = fam
        dec.close()
    return out


def run_precision(shots: int = 1 << 20, oracle_shots: int = 1 << 15, seed: int = 31):
    """Precision gap: Lottery BP + OSD-0 on the rotated d=7 surface code, 7
    noisy rounds, p = 0.012, with FP32 / FP16 / INT8 messages (2^20 shots
    each, identical shots), against the FP64 oracle on the first 2^15 shots.
    Then the d=27 space-time matrix in the form whose size Table II prints."""
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
                          "precision_d7": run_precision(), "lottery_design_space": run_policies(),
                          "check_rule": run_sum_product()}),
              flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
