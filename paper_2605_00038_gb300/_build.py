"""In-tree build of the native libraries.

* ``liblbp.so``      the decoder (CUDA, sm_103a only), from ``csrc/*.cu``.
* ``libsynth.so``    the seeded input generator (plain C), from ``inputs/``.

Compiles with nvcc / gcc directly (no cmake, no torch extension machinery),
so the same command works on the x86 build host and on an aarch64 GPU host.
A library is rebuilt only when one of its sources is newer than it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
LIBLBP = PKG / "liblbp.so"
LIBSYNTH = PKG / "inputs" / "libsynth.so"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not Path(cand).exists():
        raise RuntimeError("nvcc not found; the decoder library needs the CUDA toolkit")
    return cand


def _stale(target: Path, sources) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(s).stat().st_mtime > t for s in sources)


def _run(cmds):
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for c in cmds]
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("build failed: %s\n%s" % (" ".join(map(str, c)), out.decode(errors="replace")))


def lbp_sources():
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cuh")) + sorted(INCLUDE.glob("*.h"))


def build_lbp(force: bool = False, verbose_ptxas: bool = False) -> Path:
    srcs = lbp_sources()
    if not force and not _stale(LIBLBP, srcs):
        return LIBLBP
    nvcc = _nvcc()
    build_dir = PKG / "_build"
    build_dir.mkdir(exist_ok=True)
    units = sorted(CSRC.glob("*.cu"))
    objs = []
    cmds = []
    for u in units:
        o = build_dir / (u.stem + ".o")
        objs.append(o)
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-fmad=false", "-I", str(INCLUDE), "-I", str(CSRC), "-c", str(u), "-o", str(o)]
        if verbose_ptxas:
            cmd.insert(1, "-Xptxas=-v")
        cmds.append(cmd)
    _run(cmds)
    tmp = LIBLBP.with_suffix(".so.tmp")
    _run([[nvcc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lpthread"]])
    os.replace(tmp, LIBLBP)
    return LIBLBP


def build_synth(force: bool = False) -> Path:
    src = PKG / "inputs" / "sampler.c"
    if not force and not _stale(LIBSYNTH, [src]):
        return LIBSYNTH
    tmp = LIBSYNTH.with_suffix(".so.tmp")
    _run([["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-pthread", str(src), "-o", str(tmp)]])
    os.replace(tmp, LIBSYNTH)
    return LIBSYNTH


def build_all(force: bool = False):
    build_synth(force)
    build_lbp(force)
