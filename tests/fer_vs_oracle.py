"""FER/BER of the GPU decoder (FP32, FP16 and BF16 messages) beside the FP64
oracle on a bounded sample, with 95% Wilson intervals.

Test infrastructure (runs the oracle). Usage on a GPU machine:

    python tests/fer_vs_oracle.py --code n64800 --ebn0 1.0 1.2 1.4 \
        --gpu-frames 1000000 --oracle-seconds 240

Both sides draw the channel from Philox-4x64-10 with the same seed and
global frame indices (each side its own implementation), so the oracle's
frames are the first frames of the GPU run.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--code", default="n64800")
    p.add_argument("--ebn0", type=float, nargs="+", default=[1.0, 1.2, 1.4])
    p.add_argument("--gpu-frames", type=int, default=1000000)
    p.add_argument("--oracle-seconds", type=float, default=240.0, help="wall-clock budget per point")
    p.add_argument("--max-iter", type=int, default=50)
    p.add_argument("--seed", type=int, default=1)
    args = p.parse_args()

    from oracle import oracle
    from paper_1609_01567_gb300 import ber, ldpc

    code = ber.CODES[args.code]()
    h = ldpc.code_from_inputs(code)
    cores = os.cpu_count() or 1
    for eb in args.ebn0:
        row = {"code": args.code, "ebn0_db": eb, "max_iter": args.max_iter}
        for msg in ("f32", "f16", "bf16"):
            t0 = time.perf_counter()
            c = ber.simulate(h, code, eb, args.gpu_frames, batch=1024, max_iter=args.max_iter, msg_dtype=msg,
                             seed=args.seed)
            row[msg] = {**ber.summary(c, code.n), "seconds": round(time.perf_counter() - t0, 2)}
        # oracle: batches of one frame per core until the budget is spent
        sigma2 = ber.inputs.sigma2_from_ebn0(eb, code.rate)
        done = errs = bit_errs = iters = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < args.oracle_seconds:
            lam = oracle.gen_awgn(args.seed, done, cores, code.n, sigma2)
            out = oracle.decode(code, lam, args.max_iter, want_post=False, n_threads=cores)
            done += cores
            errs += int(out["bits"].any(axis=1).sum())
            bit_errs += int(out["bits"].sum())
            iters += int(out["iters"].sum())
        row["oracle_fp64"] = {"frames": done, "frame_errors": errs, "fer": errs / done,
                              "fer_ci95": list(ber.wilson(errs, done)), "bit_errors": bit_errs,
                              "ber": bit_errs / (done * code.n), "mean_iters": iters / done,
                              "seconds": round(time.perf_counter() - t0, 1), "cores": cores}
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
