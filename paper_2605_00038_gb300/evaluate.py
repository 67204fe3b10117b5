"""Scoring of decode results: logical failures and error-rate statistics.

A shot fails logically when BP did not converge and OSD did not replace its
estimate, or when the residual r = e xor e_hat (true error and estimate,
packed bits) is a logical operator: its data part, summed over the rounds
of a space-time matrix (one round for code capacity), anticommutes with one
of the code's logical operators L (L r_data != 0 mod 2).  This scores the
decoder's output; it is not part of decoding.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from .inputs.codes import SparseH, bb_code, logical_operators, rotated_surface, unrotated_surface


@dataclass
class LogicalSpec:
    L: np.ndarray        # [k][n_data] logical operators of one round
    rounds: int          # data blocks of the space-time matrix (1: code capacity)
    n_data: int          # columns per round
    n_total: int         # columns of the decoded matrix


def surface_spec(d: int, rounds: int, n_total: int) -> LogicalSpec:
    hz, hx = rotated_surface(d)
    return LogicalSpec(logical_operators(hz, hx), rounds, hz.n, n_total)


def unrotated_surface_spec(d: int, rounds: int, n_total: int) -> LogicalSpec:
    """Logical operators for X errors detected by the unrotated code's Z
    checks (Table III's H_Z rows), per round of a space-time matrix."""
    hx, hz = unrotated_surface(d)
    return LogicalSpec(logical_operators(hz, hx), rounds, hz.n, n_total)


def bb_spec(name: str) -> LogicalSpec:
    hx, hz = bb_code(name)
    return LogicalSpec(logical_operators(hx, hz), 1, hx.n, hx.n)


def logical_failures(spec: LogicalSpec, true_words, est_words, converged, osd_status,
                     chunk: int = 50_000) -> torch.Tensor:
    """Per-shot failure flags (bool tensor on the device of the inputs).

    true_words, est_words: [B][ceil(n/64)] int64 tensors (uint64 bit patterns);
    converged, osd_status: [B] uint8 tensors (osd_status 1 = OSD applied)."""
    dev = est_words.device
    L = torch.from_numpy(spec.L.astype(np.float32)).to(dev)
    shifts = torch.arange(64, device=dev, dtype=torch.int64)
    B = est_words.shape[0]
    out = torch.empty(B, dtype=torch.bool, device=dev)
    for lo in range(0, B, chunk):
        hi = min(B, lo + chunk)
        r = torch.bitwise_xor(true_words[lo:hi].to(dev), est_words[lo:hi])
        bits = torch.bitwise_and(torch.bitwise_right_shift(r.unsqueeze(-1), shifts), 1)
        bits = bits.reshape(hi - lo, -1)[:, : spec.n_total]
        data = bits[:, : spec.rounds * spec.n_data].reshape(hi - lo, spec.rounds, spec.n_data)
        data = data.sum(1).remainder(2).float()
        hit = (data @ L.T).remainder(2).sum(1) > 0
        unresolved = (converged[lo:hi] == 0) & (osd_status[lo:hi] != 1)
        out[lo:hi] = hit | unresolved.to(dev)
    return out


def wilson(k: int, n: int, z: float = 1.96):
    """95% Wilson score interval of a binomial proportion."""
    if n == 0:
        return (0.0, 1.0)
    p = k / n
    den = 1 + z * z / n
    c = (p + z * z / (2 * n)) / den
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return (max(0.0, c - h), min(1.0, c + h))


def mcnemar_p(b: int, c: int) -> float:
    """Two-sided exact McNemar p-value for b, c discordant pairs."""
    n = b + c
    if n == 0:
        return 1.0
    k = min(b, c)
    # P(X <= k) for X ~ Binomial(n, 1/2), doubled.
    logp = [math.lgamma(n + 1) - math.lgamma(i + 1) - math.lgamma(n - i + 1) - n * math.log(2)
            for i in range(k + 1)]
    m = max(logp)
    s = sum(math.exp(x - m) for x in logp) * math.exp(m)
    return min(1.0, 2 * s)
