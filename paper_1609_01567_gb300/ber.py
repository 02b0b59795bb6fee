"""BER/FER simulation on the GPU (the BER simulator of Section IV).

Every batch runs its library calls on one stream: the Philox BPSK/AWGN
generator (all-zero codeword, enough by linearity, or random codewords --
given, or drawn on the device from Philox information bits and the IRA
encoder), the decoder, and the on-device error count. Counters stay on the device
until the end. Frame noise depends only on (seed, global frame index), so
runs split across batches or ranks see the same channel.

    python -m paper_1609_01567_gb300.ber --code n64800 --ebn0 1.0 1.2 1.4 \
        --frames 1000000 --batch 1024 --msg f32 f16 bf16 i8
    python -m paper_1609_01567_gb300.ber --code n16200_r1/3 --ebn0 1.0 \
        --rule min_sum_adaptive --degree-alpha 1 1 1 0.94 0.88
    python -m paper_1609_01567_gb300.ber --frames 10000000 --checkpoint run.json

With --checkpoint, each point runs in chunks of --chunk-frames and its
counts and next frame index are saved after every chunk; a run started
again with the same file continues every point where it stopped. Frames are
numbered globally, so a resumed run decodes exactly the frames (and noise) an
uninterrupted one would, and gives the same counts.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import os

from . import inputs
from .shard import Counts


def wilson(k: int, n: int, z: float = 1.96) -> tuple[float, float]:
    """Wilson score interval of a binomial proportion k / n."""
    if n == 0:
        return 0.0, 1.0
    p = k / n
    den = 1 + z * z / n
    mid = (p + z * z / (2 * n)) / den
    half = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return max(0.0, mid - half), min(1.0, mid + half)


def simulate(handle, code, ebn0_db: float, n_frames: int, *, batch: int = 1024, max_iter: int = 50,
             early_exit: bool = True, msg_dtype: str = "f32", seed: int = 1, frame_offset: int = 0,
             codewords=None, stream=None, **decode_kw) -> Counts:
    """Decode n_frames noisy frames; returns summed Counts.

    codewords: None for the all-zero word, "random" for random codewords
    made on the device (information bits from Philox key (seed, 1), encoded
    by the library's IRA encoder, or by its dense systematic encoder for a
    code without the staircase, a lifted code say), else a CUDA uint8 tensor
    [n_frames, n] of transmitted codewords.
    """
    import torch

    from . import ldpc

    dev = torch.device("cuda", handle.device)
    sigma2 = inputs.sigma2_from_ebn0(ebn0_db, code.rate)
    counts = torch.zeros(4, dtype=torch.int64, device=dev)
    llr = torch.empty((batch, code.n), dtype=torch.float32, device=dev)
    out = None
    done = 0
    rand = isinstance(codewords, str)
    if rand:
        if codewords != "random":
            raise ValueError("codewords must be None, 'random' or a tensor")
        ira = ldpc.ldpc_code_info(handle)["ira_k"] >= 0
        k = code.n - code.m if ira else ldpc.ldpc_code_build_encoder(handle)
        encode = ldpc.ldpc_encode_ira if ira else ldpc.ldpc_encode
        info = torch.empty((batch, k), dtype=torch.uint8, device=dev)
        cw_buf = torch.empty((batch, code.n), dtype=torch.uint8, device=dev)
    while done < n_frames:
        b = min(batch, n_frames - done)
        if rand:
            ldpc.ldpc_gen_bits(seed, frame_offset + done, b, k, out=info[:b], device=handle.device, stream=stream)
            cw = encode(handle, info[:b], out=cw_buf[:b], stream=stream)
        else:
            cw = None if codewords is None else codewords[done:done + b]
        lb = llr[:b]
        ldpc.ldpc_gen_awgn(seed, frame_offset + done, b, code.n, sigma2, cw, out=lb, device=handle.device,
                           stream=stream)
        if out is None or out["bits"].shape[0] != b:
            out = None
        out = ldpc.ldpc_decode(handle, lb, max_iter, early_exit=early_exit, msg_dtype=msg_dtype, want_post=False,
                               out=out, stream=stream, **decode_kw)
        ldpc.ldpc_count_errors(out["bits"], cw, out["iters"], out["ok"], counts=counts, stream=stream)
        done += b
    torch.cuda.synchronize(dev)
    v = counts.cpu().tolist()
    return Counts(frames=n_frames, bit_errors=v[0], frame_errors=v[1], iterations=v[2], unsatisfied=v[3])


def summary(c: Counts, n: int) -> dict:
    fer_lo, fer_hi = wilson(c.frame_errors, c.frames)
    ber_lo, ber_hi = wilson(c.bit_errors, c.frames * n)
    return {"frames": c.frames, "frame_errors": c.frame_errors, "bit_errors": c.bit_errors,
            "fer": c.frame_errors / max(c.frames, 1), "fer_ci95": [fer_lo, fer_hi],
            "ber": c.bit_errors / max(c.frames * n, 1), "ber_ci95": [ber_lo, ber_hi],
            "mean_iters": c.iterations / max(c.frames, 1)}


CODES = {"n1008": inputs.small_code_n1008, "n64800": inputs.large_code_n64800,
         **{name: (lambda i=i: inputs.mixed_code(i)) for i, (_, _, name) in enumerate(inputs.MIXED_SPECS)}}


def load_checkpoint(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def save_checkpoint(path, state):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(state, f, indent=1, sort_keys=True)
    os.replace(tmp, path)  # a run killed mid-write keeps the previous file


def simulate_resumable(handle, code, ebn0_db, n_frames, key, state, path, chunk_frames, **kw) -> Counts:
    """simulate() over frames [0, n_frames) in chunks, continuing from the
    counts and frame index stored under ``key`` in ``state`` and saving them
    to ``path`` after every chunk (no path: plain simulate)."""
    if not path:
        return simulate(handle, code, ebn0_db, n_frames, **kw)
    entry = state.get(key, {"next_frame": 0, "counts": Counts().as_list()})
    c = Counts.from_list(entry["counts"])
    done = int(entry["next_frame"])
    while done < n_frames:
        b = min(chunk_frames, n_frames - done)
        part = simulate(handle, code, ebn0_db, b, frame_offset=done, **kw)
        c = Counts.from_list([x + y for x, y in zip(c.as_list(), part.as_list())])
        done += b
        state[key] = {"next_frame": done, "counts": c.as_list()}
        save_checkpoint(path, state)
    return c


def main(argv=None):
    p = argparse.ArgumentParser(description="GPU BER/FER simulation")
    p.add_argument("--code", choices=sorted(CODES), default="n64800")
    p.add_argument("--ebn0", type=float, nargs="+", default=[1.0, 1.2, 1.4])
    p.add_argument("--frames", type=int, default=100000)
    p.add_argument("--batch", type=int, default=1024)
    p.add_argument("--max-iter", type=int, default=50)
    p.add_argument("--msg", nargs="+", default=["f32", "f16", "bf16"])
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--rule", default="sum_product", help="sum_product, min_sum, sp_table or min_sum_adaptive")
    p.add_argument("--alpha", type=float, default=1.0, help="min-sum scale")
    p.add_argument("--beta", type=float, default=0.0, help="min-sum offset")
    p.add_argument("--degree-alpha", type=float, nargs="+", help="min_sum_adaptive: scale by check degree 0, 1, ...")
    p.add_argument("--degree-beta", type=float, nargs="+", help="min_sum_adaptive: offset by check degree 0, 1, ...")
    p.add_argument("--checkpoint", help="JSON file of per-point counts; an interrupted run resumes from it")
    p.add_argument("--chunk-frames", type=int, default=100000, help="frames between two checkpoint saves")
    args = p.parse_args(argv)

    from . import ldpc

    code = CODES[args.code]()
    h = ldpc.code_from_inputs(code)
    rule_kw = dict(rule=args.rule, rule_alpha=args.alpha, rule_beta=args.beta)
    rule_desc = {"rule": args.rule}
    if args.rule == "min_sum":
        rule_desc.update(alpha=args.alpha, beta=args.beta)
    if args.rule == "min_sum_adaptive":
        if not args.degree_alpha:
            raise SystemExit("min_sum_adaptive needs --degree-alpha")
        ldpc.ldpc_code_set_rule_table(h, args.degree_alpha, args.degree_beta)
        rule_desc.update(degree_alpha=args.degree_alpha, degree_beta=args.degree_beta)
    state = load_checkpoint(args.checkpoint)
    for eb in args.ebn0:
        for msg in args.msg:
            t0 = time.perf_counter()
            key = json.dumps({"code": args.code, "ebn0_db": eb, "msg": msg, "max_iter": args.max_iter,
                              "seed": args.seed, "batch": args.batch, **rule_desc}, sort_keys=True)
            c = simulate_resumable(h, code, eb, args.frames, key, state, args.checkpoint, args.chunk_frames,
                                   batch=args.batch, max_iter=args.max_iter, msg_dtype=msg, seed=args.seed,
                                   **rule_kw)
            line = {"code": args.code, "ebn0_db": eb, "msg_dtype": msg, "max_iter": args.max_iter, **rule_desc,
                    "seconds": time.perf_counter() - t0, **summary(c, code.n)}
            print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
