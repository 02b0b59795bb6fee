"""Builds the C-ABI library ``libldpc_gb300`` for sm_103a, in tree.

Every source under ``csrc/`` is compiled on its own (in parallel) with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and the
objects are linked into ``_build/libldpc_gb300_<machine>.so``. No CMake.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"
GENCODE = "arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def library_path() -> Path:
    return BUILD / f"libldpc_gb300_{platform.machine()}.so"


def _sources():
    return sorted(list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cpp")))


def _headers():
    return sorted(list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + list(INCLUDE.glob("*.h")))


def _compile(src: Path, obj: Path, extra: list[str]) -> None:
    cmd = [nvcc(), "-c", str(src), "-o", str(obj), "-std=c++17", "-O3", "-lineinfo", "-gencode", GENCODE,
           "-Xcompiler", "-fPIC", "-I", str(INCLUDE), "-I", str(CSRC)] + extra
    if src.suffix == ".cpp":
        cmd += ["-x", "cu"]
    subprocess.run(cmd, check=True)


def build(force: bool = False, verbose_ptxas: bool = False) -> Path:
    out = library_path()
    srcs = _sources()
    newest = max(p.stat().st_mtime for p in srcs + _headers())
    if not force and out.exists() and out.stat().st_mtime >= newest:
        return out
    BUILD.mkdir(parents=True, exist_ok=True)
    objdir = BUILD / f"obj_{platform.machine()}"
    objdir.mkdir(exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    objs = [objdir / (s.stem + ".o") for s in srcs]
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        futs = [ex.submit(_compile, s, o, extra) for s, o in zip(srcs, objs)]
        for f in futs:
            f.result()
    tmp = out.with_suffix(".so.tmp")
    subprocess.run([nvcc(), "-shared", "-gencode", GENCODE, "-o", str(tmp)] + [str(o) for o in objs], check=True)
    tmp.replace(out)
    return out


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose_ptxas="-v" in sys.argv))
