"""Builds the FP64 oracle (``ldpc_oracle.c``) into ``oracle/_build``.

TEST INFRASTRUCTURE: the oracle is only loaded by the tests, the smoke check
and the benchmark's CPU-baseline leg. Plain gcc, IEEE arithmetic (no
-ffast-math); OpenMP parallelises over independent frames only.
"""
from __future__ import annotations

import platform
import subprocess
from pathlib import Path

HERE = Path(__file__).resolve().parent
SRC = HERE / "ldpc_oracle.c"


def library_path() -> Path:
    return HERE / "_build" / f"libldpc_oracle_{platform.machine()}.so"


def build(force: bool = False) -> Path:
    out = library_path()
    if not force and out.exists() and out.stat().st_mtime >= SRC.stat().st_mtime:
        return out
    out.parent.mkdir(parents=True, exist_ok=True)
    tmp = out.with_suffix(".so.tmp")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math", str(SRC), "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    tmp.replace(out)
    return out


if __name__ == "__main__":
    print(build(force=True))
