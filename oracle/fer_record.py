"""FP64 oracle FER/BER on the first frames of the GPU's Philox channel.

Test infrastructure: this script runs only the oracle (its own Philox-4x64-10
and Box-Muller, Section IV's BPSK/AWGN channel, all-zero codeword) and writes
a record that the GPU FER test reads. The GPU's BER simulator draws frame f of
seed s from the same counter-based generator, so the oracle's frames 0..N-1
are the first N frames of every GPU run with that seed.

    python -m oracle.fer_record --ebn0 1.0 --frames 4000
    python -m oracle.fer_record --ebn0 1.2 --frames 20000

The record (oracle/records/fer_n64800_seed1.json) holds per Eb/N0 point the
frames decoded, frame and bit errors, the indices of the frames in error and
the histogram of iteration counts (max_iter 50, early exit). Runs resume:
frames already in the record are not decoded again.
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import time
from pathlib import Path

from oracle import oracle
from paper_1609_01567_gb300 import inputs

RECORD_DIR = Path(__file__).resolve().parent / "records"


def record_path(code_name: str, seed: int) -> Path:
    return RECORD_DIR / f"fer_{code_name}_seed{seed}.json"


def load(path: Path) -> dict:
    return json.loads(path.read_text()) if path.exists() else {}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--ebn0", type=float, nargs="+", required=True)
    p.add_argument("--frames", type=int, required=True)
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--max-iter", type=int, default=50)
    p.add_argument("--chunk", type=int, default=256)
    p.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    args = p.parse_args(argv)

    code = inputs.large_code_n64800()
    path = record_path("n64800", args.seed)
    RECORD_DIR.mkdir(exist_ok=True)
    rec = load(path)
    rec.setdefault("code", "ira_n64800_r1/2 (inputs.large_code_n64800, seed 64800)")
    rec.setdefault("channel", "BPSK/AWGN, all-zero codeword, Philox-4x64-10 key (seed, 0), frames 0..N-1")
    rec.setdefault("decoder", f"FP64 oracle, sum-product, l_max 20, max_iter {args.max_iter}, early exit")
    rec.setdefault("points", {})
    for eb in args.ebn0:
        key = f"{eb:.2f}"
        pt = rec["points"].setdefault(key, {"ebn0_db": eb, "frames": 0, "frame_errors": 0, "bit_errors": 0,
                                            "error_frames": [], "iters_hist": {}, "cpu_seconds": 0.0})
        sigma2 = inputs.sigma2_from_ebn0(eb, code.rate)
        while pt["frames"] < args.frames:
            b = min(args.chunk, args.frames - pt["frames"])
            f0 = pt["frames"]
            t0 = time.perf_counter()
            lam = oracle.gen_awgn(args.seed, f0, b, code.n, sigma2)
            out = oracle.decode(code, lam, args.max_iter, want_post=False, n_threads=args.threads)
            wall = time.perf_counter() - t0
            bad = out["bits"].any(axis=1)
            pt["frame_errors"] += int(bad.sum())
            pt["bit_errors"] += int(out["bits"].sum())
            pt["error_frames"] += [int(f0 + i) for i in bad.nonzero()[0]]
            hist = collections.Counter(pt["iters_hist"])
            hist.update({str(int(k)): int(v) for k, v in collections.Counter(out["iters"].tolist()).items()})
            pt["iters_hist"] = dict(sorted(hist.items(), key=lambda kv: int(kv[0])))
            pt["frames"] += b
            pt["cpu_seconds"] = round(pt["cpu_seconds"] + wall * args.threads, 1)
            pt["threads"] = args.threads
            tmp = path.with_suffix(".tmp")
            tmp.write_text(json.dumps(rec, indent=1))
            tmp.replace(path)
            print(f"{eb} dB: {pt['frames']} frames, {pt['frame_errors']} frame errors", flush=True)


if __name__ == "__main__":
    main()
