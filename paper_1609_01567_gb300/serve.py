"""Serving benchmark: Poisson request arrivals against the decode server.

Requests carry 1..512 frames (log-uniform) of one of nine codes (the eight
mixed-workload codes and the n = 64800 rate-1/2 code), each at its
Eb/N0 of FER ~1e-2 (1.2 dB for the n = 64800 code), max_iter 50 with early
exit. Two ways to serve the same trace:

* server: ``ldpc_server`` (continuous batching over several slots), FP16
  messages; latency = submit (at the arrival time) to completion;
* plain: one FP32 ``ldpc_decode`` per request on one stream, in arrival
  order; latency = arrival to completion (queueing included).

    python -m paper_1609_01567_gb300.serve --rate 2000 --requests 3000
"""
from __future__ import annotations

import argparse
import json
import math
import threading
import time

import numpy as np

from . import inputs
from .mixed import EBN0_AT_FER_1E2

POOL_FRAMES = 2048


def serving_codes():
    codes = inputs.mixed_codes() + [inputs.large_code_n64800()]
    ebn0 = [EBN0_AT_FER_1E2[c.name] for c in codes[:-1]] + [1.2]
    return codes, ebn0


def trace(n_requests: int, rate: float, n_codes: int, seed: int = 11, max_frames: int = 512):
    """(arrival seconds, code index, frames, pool offset) per request."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    frames = np.floor(np.exp(rng.uniform(0.0, math.log(max_frames + 1), size=n_requests))).astype(int)
    frames = np.clip(frames, 1, max_frames)
    codes = rng.integers(0, n_codes, size=n_requests)
    offsets = rng.integers(0, POOL_FRAMES - max_frames, size=n_requests)
    return arrivals, codes, frames, offsets


def make_pools(codes, ebn0, device=0, seed=21):
    import torch

    from . import ldpc

    pools = []
    for i, (c, eb) in enumerate(zip(codes, ebn0)):
        cw = torch.from_numpy(inputs.encode_ira(c, inputs.random_info(POOL_FRAMES, c.k, seed=seed + i))).cuda(device)
        s2 = inputs.sigma2_from_ebn0(eb, c.rate)
        pools.append((ldpc.ldpc_gen_awgn(seed + i, 0, POOL_FRAMES, c.n, s2, cw, device=device), cw))
    return pools


def pct(x, q):
    return float(np.percentile(np.asarray(x), q)) if len(x) else None


def run_server(handles, pools, tr, msg="f16", max_slots=4, max_batch=1024):
    from . import ldpc

    arrivals, codes, frames, offsets = tr
    srv = ldpc.ldpc_server_create(handles, max_batch_frames=max_batch, max_slots=max_slots, msg_dtype=msg)
    ids = [None] * len(arrivals)
    t0 = time.perf_counter() + 0.05

    def submitter():
        for i in range(len(arrivals)):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            llr = pools[codes[i]][0][offsets[i]:offsets[i] + frames[i]]
            while True:
                try:
                    ids[i] = ldpc.ldpc_server_submit(srv, int(codes[i]), llr)
                    break
                except ldpc.LdpcError as e:
                    if e.status != -6:
                        raise
                    time.sleep(1e-4)

    th = threading.Thread(target=submitter)
    th.start()
    lat = []
    for i in range(len(arrivals)):
        while ids[i] is None:
            time.sleep(1e-4)
        lat.append(ldpc.ldpc_server_wait(srv, ids[i][0]))
    t_end = time.perf_counter()
    th.join()
    stats = ldpc.ldpc_server_stats(srv)
    srv.close()
    return lat, t_end - t0, stats


def run_plain(handles, pools, tr):
    import torch

    from . import ldpc

    arrivals, codes, frames, offsets = tr
    stream = torch.cuda.current_stream()
    start = torch.cuda.Event(enable_timing=True)
    evs = []
    t0 = time.perf_counter() + 0.05
    while time.perf_counter() < t0:
        pass
    start.record(stream)
    for i in range(len(arrivals)):
        delay = t0 + arrivals[i] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        llr = pools[codes[i]][0][offsets[i]:offsets[i] + frames[i]]
        ldpc.ldpc_decode(handles[codes[i]], llr, 50, want_post=False, streams=1)
        ev = torch.cuda.Event(enable_timing=True)
        ev.record(stream)
        evs.append(ev)
    torch.cuda.synchronize()
    done = np.array([start.elapsed_time(e) / 1e3 for e in evs])
    lat = (done - arrivals) * 1e3
    return list(lat), float(done.max())


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--rate", type=float, nargs="+", default=[2000.0])
    p.add_argument("--requests", type=int, default=3000)
    p.add_argument("--slots", type=int, default=4)
    p.add_argument("--msg", default="f16")
    p.add_argument("--no-plain", action="store_true")
    args = p.parse_args(argv)

    import torch  # noqa: F401

    from . import ldpc

    for line in measure(args.rate, args.requests, msg=args.msg, slots=args.slots, plain=not args.no_plain):
        print(json.dumps(line), flush=True)


def measure(rates, requests, msg="f16", slots=4, plain=True, device=0):
    """One Poisson trace per offered rate through the server, and (plain)
    through the per-request FP32 decoder; yields one record per rate."""
    from . import ldpc

    codes, ebn0 = serving_codes()
    handles = [ldpc.code_from_inputs(c, device=device) for c in codes]
    pools = make_pools(codes, ebn0, device=device)
    for rate in rates:
        tr = trace(requests, rate, len(codes))
        info_bits = int(sum(codes[c].k * f for c, f in zip(tr[1], tr[2])))
        lat, span, stats = run_server(handles, pools, tr, msg=msg, max_slots=slots)
        line = {"rate_req_s": rate, "requests": requests, "frames": int(tr[2].sum()), "info_bits": info_bits,
                "server": {"msg_dtype": msg, "slots": stats["slots"], "batches": stats["batches"],
                           "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "gbps": info_bits / span / 1e9,
                           "seconds": span}}
        if plain:
            lat_p, span_p = run_plain(handles, pools, tr)
            line["plain_f32"] = {"p50_ms": pct(lat_p, 50), "p99_ms": pct(lat_p, 99), "gbps": info_bits / span_p / 1e9,
                                 "seconds": span_p}
        yield line


if __name__ == "__main__":
    main()
