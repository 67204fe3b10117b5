"""CPU oracle for Lottery BP (+ OSD-0): test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
decoder (``paper_2605_00038_gb300``) and neither imports the other.
"""
from .oracle import (OracleParams, build, decode, osd0, lottery_select, splitmix64_at,
                     round_f16, round_i8, PREC_F64, PREC_F32, PREC_F16, PREC_I8)

__all__ = ["OracleParams", "build", "decode", "osd0", "lottery_select", "splitmix64_at",
           "round_f16", "round_i8", "PREC_F64", "PREC_F32", "PREC_F16", "PREC_I8"]
