"""Shared comparison rules of the GPU-vs-oracle parity tests.

Tolerance (stated for the FP32 path): a posterior LLR matches when
|gpu - oracle| <= 1e-4 |oracle| + 1e-5. Decisions and iteration counts must
match exactly, except on frames where an oracle posterior lies within that
tolerance of 0 (the sign there is a rounding coin flip); those frames are
returned so the caller can log them.
"""
from __future__ import annotations

import numpy as np

RTOL = 1e-4
ATOL = 1e-5


def close(gpu, ref, rtol=RTOL, atol=ATOL):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(gpu - ref) <= rtol * np.abs(ref) + atol


def near_zero_frames(ref_post, rtol=RTOL, atol=ATOL):
    a = np.abs(np.asarray(ref_post, dtype=np.float64))
    return np.any(a <= rtol * a + atol, axis=1)


def compare_decodes(gpu: dict, ref: dict, frames=None):
    """Per-frame verdict of a GPU decode against the oracle on the same LLRs.

    Returns (bad_frames, exempt_frames) as index arrays: bad frames have a
    posterior outside tolerance or a different decision, iteration count or
    syndrome flag while no posterior is near 0.
    """
    post_ok = close(gpu["post"], ref["post"]).all(axis=1)
    same = ((gpu["bits"] == ref["bits"]).all(axis=1) & (gpu["iters"] == ref["iters"]) & (gpu["ok"] == ref["ok"]))
    exempt = near_zero_frames(ref["post"])
    bad = ~(post_ok & same) & ~exempt
    idx = np.arange(len(bad)) if frames is None else np.asarray(frames)
    return idx[bad], idx[exempt]


def gf2_information_positions(m, n, rows, cols):
    """Column j of H is an information position iff it lies in the span of
    the columns to its right (GF(2)); independent of the library's
    elimination: a column-by-column basis of those columns, numpy bool rows."""
    H = np.zeros((m, n), dtype=bool)
    H[np.asarray(rows), np.asarray(cols)] = True
    basis = {}  # leading row -> reduced column vector
    info = []
    for j in range(n - 1, -1, -1):
        v = H[:, j].copy()
        for lead in sorted(basis):
            if v[lead]:
                v ^= basis[lead]
        nz = np.flatnonzero(v)
        if nz.size == 0:
            info.append(j)
        else:
            lead = int(nz[0])
            for key in list(basis):
                if basis[key][lead]:
                    basis[key] ^= v
            basis[lead] = v
    return sorted(info), len(basis)
