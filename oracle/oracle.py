"""ctypes front end of ``oracle.c`` (test infrastructure only).

The arrays passed in are plain numpy arrays: H in CSR form, priors p_v,
syndromes as 0/1 bytes.  Nothing here decodes; every step of the method is
in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
LIB = HERE / "liboracle.so"

PREC_F64, PREC_F32, PREC_F16, PREC_I8 = 0, 1, 2, 3
RULE_MIN_SUM, RULE_SUM_PRODUCT = 0, 1


def build(force: bool = False) -> Path:
    """Compile liboracle.so in place (gcc, no FMA contraction)."""
    if not force and LIB.exists() and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = LIB.with_suffix(".so.tmp")
    subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                    "-shared", "-fPIC", "-pthread", str(SRC), "-o", str(tmp), "-lm"],
                   check=True)
    os.replace(tmp, LIB)
    return LIB


class _Params(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int32), ("scale_mode", ctypes.c_int32),
                ("scale_const", ctypes.c_double), ("lottery", ctypes.c_int32),
                ("lottery_skip", ctypes.c_int32), ("osd", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("early_exit", ctypes.c_int32),
                ("rule", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("shot_offset", ctypes.c_uint64)]


@dataclass
class OracleParams:
    max_iter: int = 100
    scale_mode: int = 1          # 0 constant, 1 adaptive 1 - 2^-(i+1)
    scale_const: float = 0.625
    lottery: bool = True
    lottery_skip: int = 6
    osd: bool = False
    prec: int = PREC_F64
    early_exit: bool = True
    rule: int = RULE_MIN_SUM
    policy: int = 0              # lottery policy: 0 proposed, 1..4 baselines (Sec. III-B), 5 ablation (U from s_hat(i))
    seed: int = 0
    shot_offset: int = 0

    def _c(self) -> _Params:
        return _Params(self.max_iter, self.scale_mode, self.scale_const, int(self.lottery),
                       self.lottery_skip, int(self.osd), self.prec, int(self.early_exit),
                       self.rule, self.policy, self.seed, self.shot_offset)


_L = None


def _lib():
    global _L
    if _L is None:
        if not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
            build()
        lib = ctypes.CDLL(str(LIB))
        vp = ctypes.c_void_p
        lib.oracle_decode.restype = ctypes.c_int
        lib.oracle_decode.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                      ctypes.POINTER(_Params), ctypes.c_int64,
                                      vp, vp, vp, vp, vp, vp, vp, ctypes.c_int]
        lib.oracle_osd0.restype = ctypes.c_int
        lib.oracle_osd0.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
        lib.oracle_lottery_select.restype = ctypes.c_int
        lib.oracle_lottery_select.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp,
                                              ctypes.c_uint64, ctypes.c_int, vp, vp]
        lib.oracle_splitmix64_at.restype = ctypes.c_uint64
        lib.oracle_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_round_f16.restype = ctypes.c_double
        lib.oracle_round_f16.argtypes = [ctypes.c_double]
        lib.oracle_round_i8.restype = ctypes.c_double
        lib.oracle_round_i8.argtypes = [ctypes.c_double]
        _L = lib
    return _L


def _csr(h):
    return (np.ascontiguousarray(h.row_ptr, dtype=np.int32),
            np.ascontiguousarray(h.col_idx, dtype=np.int32))


def _ptr(a):
    return None if a is None else a.ctypes.data


@dataclass
class DecodeResult:
    err: np.ndarray        # [B][n] uint8
    converged: np.ndarray  # [B] uint8
    osd_used: np.ndarray   # [B] uint8
    osd_nosol: np.ndarray  # [B] uint8
    iters: np.ndarray      # [B] int32
    llr: np.ndarray | None  # [B][n] float64


def decode(h, priors, syndromes, params: OracleParams, want_llr: bool = False,
           nthreads: int | None = None) -> DecodeResult:
    """Decode syndromes ([B][m] 0/1 array) on the CPU, shot by shot."""
    rp, ci = _csr(h)
    pri = np.ascontiguousarray(priors, dtype=np.float64)
    syn = np.ascontiguousarray(syndromes, dtype=np.uint8)
    if syn.ndim != 2 or syn.shape[1] != h.m or pri.shape != (h.n,):
        raise ValueError("shape mismatch")
    B = syn.shape[0]
    err = np.zeros((B, h.n), dtype=np.uint8)
    conv = np.zeros(B, dtype=np.uint8)
    used = np.zeros(B, dtype=np.uint8)
    nosol = np.zeros(B, dtype=np.uint8)
    iters = np.zeros(B, dtype=np.int32)
    llr = np.zeros((B, h.n), dtype=np.float64) if want_llr else None
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    prm = params._c()
    rc = _lib().oracle_decode(h.m, h.n, _ptr(rp), _ptr(ci), _ptr(pri), ctypes.byref(prm), B,
                              _ptr(syn), _ptr(err), _ptr(conv), _ptr(used), _ptr(nosol),
                              _ptr(iters), _ptr(llr), nthreads)
    if rc != 0:
        raise ValueError("oracle_decode rejected its input (code %d)" % rc)
    return DecodeResult(err, conv, used, nosol, iters, llr)


def osd0(h, llr, s):
    """OSD-0 of one shot: returns (e [n] uint8 or None if no solution, rank, basis)."""
    rp, ci = _csr(h)
    lam = np.ascontiguousarray(llr, dtype=np.float64)
    sv = np.ascontiguousarray(s, dtype=np.uint8)
    e = np.zeros(h.n, dtype=np.uint8)
    rank = ctypes.c_int32(0)
    basis = np.zeros(max(h.m, 1), dtype=np.int32)
    rc = _lib().oracle_osd0(h.m, h.n, _ptr(rp), _ptr(ci), _ptr(lam), _ptr(sv), _ptr(e),
                            ctypes.addressof(rank), _ptr(basis))
    if rc < 0:
        raise ValueError("oracle_osd0 rejected its input (code %d)" % rc)
    return (e if rc == 0 else None), rank.value, basis[:rank.value].copy()


def lottery_select(h, U, llr, u: int, policy: int = 0):
    """Lottery selection for one shot: returns (c*, v*).  u is the 64-bit draw
    (low 32 bits: random check; high 32 bits: random column)."""
    rp, ci = _csr(h)
    Ub = np.ascontiguousarray(U, dtype=np.uint8)
    lam = np.ascontiguousarray(llr, dtype=np.float64)
    cs = ctypes.c_int32(-1)
    vs = ctypes.c_int32(-1)
    rc = _lib().oracle_lottery_select(h.m, h.n, _ptr(rp), _ptr(ci), _ptr(Ub), _ptr(lam), u, policy,
                                      ctypes.addressof(cs), ctypes.addressof(vs))
    if rc != 0:
        raise ValueError("oracle_lottery_select rejected its input (code %d)" % rc)
    return cs.value, vs.value


def splitmix64_at(seed: int, counter: int) -> int:
    return int(_lib().oracle_splitmix64_at(seed, counter))


def round_f16(x: float) -> float:
    return float(_lib().oracle_round_f16(x))


def round_i8(x: float) -> float:
    return float(_lib().oracle_round_i8(x))
