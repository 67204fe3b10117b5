"""Synthetic workload recipes (code, noise, shot count, seed, decoder settings).

The paper samples circuit-level noise with Stim, which is not available; these
seeded stand-ins keep the shapes and noise levels of the evaluated decoders:
i.i.d. Bernoulli(p) flips on every column of H (code capacity) or of the
space-time matrix (phenomenological noise, data and measurement flips).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .codes import SparseH, bb_code, block_diag, rotated_surface, spacetime, spacetime_priors


@dataclass
class Workload:
    name: str
    h: SparseH
    priors: np.ndarray
    shots: int
    seed: int
    decoder: dict = field(default_factory=dict)   # lbp_params fields
    describe: str = ""


def c1_d3_code_capacity() -> Workload:
    hz, _ = rotated_surface(3)
    return Workload("rotated_d3_cc_p0.05", hz, np.full(hz.n, 0.05), 10_000, 1,
                    dict(max_iter=20, scale_mode=0, scale_const=0.625, lottery=0, osd=0, msg=0),
                    "rotated surface d=3, H_Z 4x9, code capacity p=0.05, plain NMS f=0.625, I=20")


def c2_d11_spacetime(shots: int = 1_000_000, osd: int = 1) -> Workload:
    hz, _ = rotated_surface(11)
    st = spacetime(hz, 11)
    return Workload("rotated_d11_st11_p0.003", st, spacetime_priors(hz, 11, 0.003, 0.003), shots, 2,
                    dict(max_iter=100, scale_mode=1, lottery=1, lottery_skip=6, osd=osd, msg=0),
                    "rotated surface d=11, 11 rounds space-time H 660x1931 (nnz 3620), "
                    "p_data=p_meas=0.003, Lottery BP I=100 + OSD-0, FP32 messages")


def c3_bb144(p: float, shots: int = 1_000_000) -> Workload:
    hx, _ = bb_code("bb144")
    seed = {0.01: 3, 0.03: 4, 0.05: 5}.get(p, 3)
    return Workload("bb144_cc_p%g" % p, hx, np.full(hx.n, p), shots, seed,
                    dict(max_iter=100, scale_mode=1, lottery=1, lottery_skip=6, osd=1, msg=1),
                    "BB [[144,12,12]] H_X=[A|B] 72x144, code capacity p=%g, Lottery BP + OSD-0, "
                    "FP16 messages" % p)


def c5_d25_spacetime(msg: int = 0, shots: int = 1 << 20) -> Workload:
    hz, _ = rotated_surface(25)
    st = spacetime(hz, 25)
    return Workload("rotated_d25_st25_p0.004", st, spacetime_priors(hz, 25, 0.004, 0.004), shots, 6,
                    dict(max_iter=100, scale_mode=1, lottery=1, lottery_skip=6, osd=0, msg=msg),
                    "rotated surface d=25, 25 rounds space-time H 7800x23113 (nnz 44976), p=0.004")


def c5_d25_spacetime_xz(msg: int = 0, shots: int = 1 << 20) -> Workload:
    """The stress form of the d=25 workload: X and Z space-time matrices on the
    block diagonal (both error types decoded in one call), 15,600 x 46,226."""
    hx, hz = rotated_surface(25)
    st = block_diag(spacetime(hz, 25), spacetime(hx, 25))
    pri = np.concatenate([spacetime_priors(hz, 25, 0.004, 0.004), spacetime_priors(hx, 25, 0.004, 0.004)])
    return Workload("rotated_d25_st25_xz_p0.004", st, pri, shots, 7,
                    dict(max_iter=100, scale_mode=1, lottery=1, lottery_skip=6, osd=0, msg=msg),
                    "rotated surface d=25, 25 rounds, X and Z space-time H block-diagonal 15600x46226, p=0.004")


def serving_codes():
    """The ten codes of the serving mix: surface H_st d = 5..17 (d rounds) and
    BB 72 / 144 / 288 code capacity."""
    out = []
    for d in (5, 7, 9, 11, 13, 15, 17):
        hz, _ = rotated_surface(d)
        out.append(("surface_d%d_st" % d, spacetime(hz, d), (hz, d)))
    for name in ("bb72", "bb144", "bb288"):
        hx, _ = bb_code(name)
        out.append((name, hx, None))
    return out
