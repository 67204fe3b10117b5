"""Python side of the seeded input generator (see ``sampler.c``)."""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .codes import SparseH

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        from .._build import LIBSYNTH, build_synth
        if not LIBSYNTH.exists():
            build_synth()
        lib = ctypes.CDLL(str(LIBSYNTH))
        lib.synth_sample.restype = ctypes.c_int
        lib.synth_sample.argtypes = [
            ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int]
        lib.synth_splitmix64_at.restype = ctypes.c_uint64
        lib.synth_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        _LIB = lib
    return _LIB


def words(bits: int) -> int:
    return (bits + 63) // 64


def thresholds(priors: np.ndarray) -> np.ndarray:
    """floor(p * 2^32) per column, the Bernoulli cut of the sampler."""
    p = np.asarray(priors, dtype=np.float64)
    if np.any(p < 0) or np.any(p >= 1):
        raise ValueError("priors must lie in [0, 1)")
    return np.floor(p * 4294967296.0).astype(np.uint64).clip(0, 0xFFFFFFFF).astype(np.uint32)


def sample(h: SparseH, priors, seed: int, num_shots: int, shot_offset: int = 0,
           with_errors: bool = True, nthreads: int | None = None):
    """Return (errors [B][ceil(n/64)] u64 or None, syndromes [B][ceil(m/64)] u64)."""
    col_ptr, row_idx = h.csc()
    col_ptr = np.ascontiguousarray(col_ptr, dtype=np.int32)
    row_idx = np.ascontiguousarray(row_idx, dtype=np.int32)
    thr = np.ascontiguousarray(thresholds(priors))
    if thr.shape[0] != h.n:
        raise ValueError("one prior per column")
    syn = np.zeros((num_shots, words(h.m)), dtype=np.uint64)
    err = np.zeros((num_shots, words(h.n)), dtype=np.uint64) if with_errors else None
    if nthreads is None:
        nthreads = min(64, os.cpu_count() or 1)
    rc = _lib().synth_sample(h.m, h.n, col_ptr.ctypes.data, row_idx.ctypes.data, thr.ctypes.data,
                             seed, shot_offset, num_shots,
                             err.ctypes.data if err is not None else None, syn.ctypes.data, nthreads)
    if rc != 0:
        raise RuntimeError("synth_sample failed")
    return err, syn


def splitmix64_at(seed: int, counter: int) -> int:
    return int(_lib().synth_splitmix64_at(seed, counter))


def unpack(words_arr: np.ndarray, bits: int) -> np.ndarray:
    """[B][W] u64 little-endian words -> [B][bits] uint8."""
    a = np.ascontiguousarray(words_arr, dtype=np.uint64)
    b = np.unpackbits(a.view(np.uint8), axis=-1, bitorder="little")
    return b[..., :bits]


def pack(bits_arr: np.ndarray) -> np.ndarray:
    """[B][bits] 0/1 -> [B][ceil(bits/64)] u64 little-endian words."""
    a = np.asarray(bits_arr, dtype=np.uint8)
    nb = a.shape[-1]
    w = words(nb)
    pad = np.zeros(a.shape[:-1] + (w * 64,), dtype=np.uint8)
    pad[..., :nb] = a
    return np.packbits(pad, axis=-1, bitorder="little").view(np.uint64)
