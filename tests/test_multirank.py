"""Multi-rank sharding on CPU ranks (gloo, world size 2).

Each rank takes its contiguous share of the frames, draws their channel LLRs
from their global frame indices, decodes them (here with the CPU oracle,
since these ranks have no GPU) and the counters are summed with all_reduce.
The totals must equal one process decoding every frame.
"""
import os
import socket

import numpy as np

from paper_1609_01567_gb300 import inputs as I
from paper_1609_01567_gb300.shard import Counts, frame_range

TOTAL = 37
EBN0 = 1.5
MAX_ITER = 12


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def decode_range(start, count):
    from oracle import oracle

    code = I.small_code_n1008()
    cw = I.encode_ira(code, I.random_info(TOTAL, code.k, seed=3))[start:start + count]
    s2 = I.sigma2_from_ebn0(EBN0, code.rate)
    lam = oracle.gen_awgn(5, start, count, code.n, s2, cw)
    out = oracle.decode(code, lam, MAX_ITER, want_post=False)
    c = Counts()
    c.add_decode(out["bits"], out["iters"], out["ok"], cw)
    return c


def worker(rank, world, port, result_path):
    import torch.distributed as dist

    from paper_1609_01567_gb300.shard import allreduce_counts

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        start, count = frame_range(TOTAL, world, rank)
        total = allreduce_counts(decode_range(start, count))
        if rank == 0:
            np.save(result_path, np.array(total.as_list(), dtype=np.int64))
    finally:
        dist.destroy_process_group()


def test_frame_ranges_cover_every_frame_once():
    for total in (0, 1, 7, 256, 1001):
        for world in (1, 2, 3, 8):
            seen = []
            for rank in range(world):
                start, count = frame_range(total, world, rank)
                seen.extend(range(start, start + count))
            assert seen == list(range(total))


def test_two_gloo_ranks_equal_one_process(tmp_path):
    import torch.multiprocessing as mp

    result = tmp_path / "totals.npy"
    mp.start_processes(worker, args=(2, free_port(), str(result)), nprocs=2, join=True, start_method="spawn")
    sharded = np.load(result)
    single = decode_range(0, TOTAL).as_list()
    np.testing.assert_array_equal(sharded, single)
    assert single[0] == TOTAL
