"""Mixed-code batch workload: eight codes, Zipf-split frames, one CUDA graph.

4096 frames split over the eight codes of ``inputs.mixed_codes()`` by
Zipf(1.1) (shortest code most), each code at the Eb/N0 where its frame error
rate is about 1e-2, max_iter 50 with per-frame syndrome exit. Compares

* plain: one ``ldpc_decode`` per code with FP32 messages, one after another;
* batch: every code as a branch of one captured CUDA graph
  (``ldpc_batch_run``), schedules autotuned per code, FP32 or BF16 messages.

    python -m paper_1609_01567_gb300.mixed --calibrate       # Eb/N0 at FER ~1e-2
    python -m paper_1609_01567_gb300.mixed --bench --reps 20
"""
from __future__ import annotations

import argparse
import json
import time

from . import inputs

TOTAL_FRAMES = 4096
# Eb/N0 (dB) at which each mixed code's FER is about 1e-2 (FP32 messages,
# max_iter 50, early exit; bisection over 4000 frames per point), from
# `--calibrate` on a GB300.
EBN0_AT_FER_1E2 = {
    "n576_r5/6": 4.15,
    "n1152_r3/4": 3.21,
    "n2304_r2/3": 2.52,
    "n4096_r1/2": 1.7,
    "n8192_r3/4_deg64_96": 2.56,
    "n16200_r1/3": 1.25,
    "n32400_r2/3": 1.93,
    "n64800_r5/6": 2.97,
}


def workload():
    codes = inputs.mixed_codes()
    frames = inputs.zipf_frames(TOTAL_FRAMES, len(codes))
    return codes, frames


def calibrate(handle, code, target: float = 1e-2, frames: int = 4000, lo: float = 0.0, hi: float = 7.0,
              steps: int = 9) -> float:
    """Bisection on Eb/N0 for FER ~= target (FP32 messages, max_iter 50)."""
    from . import ber

    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        c = ber.simulate(handle, code, mid, frames, batch=min(frames, 2048), max_iter=50)
        if c.frame_errors / c.frames > target:
            lo = mid
        else:
            hi = mid
    return round(0.5 * (lo + hi), 2)


def make_llrs(codes, frames, seed: int = 7, device: int = 0):
    """Channel LLRs of random codewords per code at its calibrated Eb/N0."""
    import torch

    from . import ldpc

    llrs, sent = [], []
    for i, (c, f) in enumerate(zip(codes, frames)):
        cw = torch.from_numpy(inputs.encode_ira(c, inputs.random_info(f, c.k, seed=seed + i))).cuda(device)
        s2 = inputs.sigma2_from_ebn0(EBN0_AT_FER_1E2[c.name], c.rate)
        llrs.append(ldpc.ldpc_gen_awgn(seed + i, 0, f, c.n, s2, cw, device=device))
        sent.append(cw)
    return llrs, sent


def bench(reps: int = 20, device: int = 0) -> dict:
    import torch

    from . import ldpc

    codes, frames = workload()
    handles = [ldpc.code_from_inputs(c, device=device) for c in codes]
    llrs, sent = make_llrs(codes, frames, device=device)
    info_bits = sum(c.k * f for c, f in zip(codes, frames))
    result = {"frames": frames, "codes": [c.name for c in codes], "info_bits_per_run": info_bits}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            fn()
        t1.record()
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / reps

    outs = [None] * len(codes)

    def plain():
        for i, (h, l) in enumerate(zip(handles, llrs)):
            outs[i] = ldpc.ldpc_decode(h, l, 50, want_post=False, out=outs[i], streams=1)

    ms = timed(plain)
    fe = [int((o["bits"] != s).any(dim=1).sum()) for o, s in zip(outs, sent)]
    result["plain_f32"] = {"ms": ms, "gbps": info_bits / (ms * 1e-3) / 1e9, "frame_errors": fe}
    for msg in ("f32", "bf16"):
        b = ldpc.ldpc_batch_create(handles, frames, 50, msg_dtype=msg)
        ldpc.ldpc_batch_tune(b, llrs)
        bouts = ldpc.ldpc_batch_run(b, llrs)
        ms = timed(lambda: ldpc.ldpc_batch_run(b, llrs, bouts))
        fe = [int((o["bits"] != s).any(dim=1).sum()) for o, s in zip(bouts, sent)]
        sched = [ldpc.ldpc_batch_info(b, i) for i in range(len(codes))]
        result[f"batch_graph_{msg}"] = {"ms": ms, "gbps": info_bits / (ms * 1e-3) / 1e9, "frame_errors": fe,
                                        "schedules": [(s["frames_per_lane"], s["check_schedule"], s["streams"]) for s in sched],
                                        "kernels_per_run": sched[0]["kernels_per_run"]}
        b.close()
    return result


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--calibrate", action="store_true")
    p.add_argument("--bench", action="store_true")
    p.add_argument("--reps", type=int, default=20)
    args = p.parse_args(argv)
    from . import ldpc

    if args.calibrate:
        for c in inputs.mixed_codes():
            h = ldpc.code_from_inputs(c)
            print(json.dumps({"code": c.name, "ebn0_db_at_fer_1e-2": calibrate(h, c)}), flush=True)
    if args.bench:
        t0 = time.perf_counter()
        r = bench(args.reps)
        r["wall_s"] = time.perf_counter() - t0
        print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
