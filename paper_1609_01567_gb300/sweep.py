"""The paper's benchmark form (Table 3) on synthetic stand-in codes.

The paper times a BER simulation of 10,000 codewords at Eb/N0 = 2 dB for
rate-1/2 codes of n = 2^8 .. 2^18 bits with 4 edges per bit (noise
generation included), on a Tesla K40/K80 and a Xeon E5-2695v2. Its codes
(CCSDS (256,128) and protograph expansions) are not available here, so each
length gets a seeded stand-in with the same size and edge count: an IRA
code (information bits of degree 6, the staircase parity bits of degree 2:
E = 4n - 1), or, with --family qc, a (4, 8)-regular quasi-cyclic code lifted
from an all-ones 4 x 8 protograph with seeded circulant shifts (E = 4n), the
structure of the paper's protograph expansions. Per length: the on-device Philox generator, the decoder
(max_iter 50, early exit) and the error counter, all on one stream; the
paper's seconds are printed beside as context (other hardware, other codes,
unstated iteration limit).

    python -m paper_1609_01567_gb300.sweep --frames 10000
"""
from __future__ import annotations

import argparse
import json
import time

from . import inputs

# Table 3: seconds for 10,000 codewords at 2 dB -- (CUDA on the K40/K80, C++ with -O3 on the Xeon).
PAPER_TABLE3_SECONDS = {
    256: (0.32, 3.11),
    512: (0.61, 6.24),
    1024: (1.24, 12.52),
    2048: (2.51, 25.27),
    4096: (5.46, 69.17),
    8192: (12.08, 172.67),
    16384: (26.08, 367.75),
    32768: (56.02, 1025.9),
    65536: (116.86, 1989.26),
    131072: (242.43, 5215.11),
    262144: (498.16, 12287.61),
}


def stand_in_code(n: int) -> inputs.Code:
    """Seeded rate-1/2 IRA code with about 4 edges per bit."""
    return inputs.ira_code(n, n // 2, {6: 1.0}, seed=n, name=f"ira_n{n}_r1/2_4epb")


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--frames", type=int, default=10000)
    p.add_argument("--ebn0", type=float, default=2.0)
    p.add_argument("--max-iter", type=int, default=50)
    p.add_argument("--lengths", type=int, nargs="+", default=sorted(PAPER_TABLE3_SECONDS))
    p.add_argument("--msg", default="f32")
    p.add_argument("--family", choices=("ira", "qc"), default="ira")
    args = p.parse_args(argv)

    import torch

    from . import ber, ldpc

    for n in args.lengths:
        if args.family == "qc":
            code, entries = inputs.qc_stand_in_code(n)
            h = ldpc.ldpc_code_create_qc(4, 8, n // 8, entries)
        else:
            code = stand_in_code(n)
            h = ldpc.code_from_inputs(code)
        batch = max(256, min(args.frames, (1 << 31) // (16 * code.n_edges)))
        ber.simulate(h, code, args.ebn0, min(batch, args.frames), batch=batch, max_iter=args.max_iter,
                     msg_dtype=args.msg, seed=99)  # warm-up (workspace, kernel set-up)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c = ber.simulate(h, code, args.ebn0, args.frames, batch=batch, max_iter=args.max_iter, msg_dtype=args.msg,
                         seed=1)
        sec = time.perf_counter() - t0
        paper_cuda, paper_cpu = PAPER_TABLE3_SECONDS.get(n, (None, None))
        print(json.dumps({"n": n, "family": args.family, "code": code.name, "edges": code.n_edges, "frames": args.frames, "ebn0_db": args.ebn0,
                          "max_iter": args.max_iter, "msg_dtype": args.msg, "batch": batch, "seconds": sec,
                          "frames_per_s": args.frames / sec, "info_gbps": args.frames * (n // 2) / sec / 1e9,
                          **ber.summary(c, n), "paper_cuda_seconds": paper_cuda, "paper_cpu_o3_seconds": paper_cpu,
                          "speedup_vs_paper_cuda": paper_cuda / sec if paper_cuda else None}), flush=True)
        h.close()


if __name__ == "__main__":
    main()
