"""Parity at the benchmark's own workload: the n = 64800, rate-1/2 code.

The benchmark times ldpc_decode on 256 frames, max_iter 10 fixed, FP32
messages, hard decisions without posteriors, in the library's default launch
configuration (two streams, four frames per lane). These tests run exactly
that call on every one of the 256 frames against the FP64 oracle, and the
workload's second form (max_iter 50 with per-frame early exit, Algorithm 2)
on frames spread over both stream halves and several 128-frame groups.

Inputs: the same information words and Philox noise realisation as the
benchmark's first LLR buffer, drawn by the oracle's own Philox-4x64-10 and
Box-Muller in FP64 and rounded to float once, so no input comes from the CUDA
path. Rule (stated for the FP32 path): decisions, iteration counts and
syndrome flags exact, except frames with an oracle posterior within the
posterior tolerance of 0 (logged); posteriors within 1e-4 relative + 1e-5
absolute.
"""
import os

import numpy as np
import pytest

from paper_1609_01567_gb300 import inputs as I
from tests.parity import close, near_zero_frames

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BENCH_FRAMES = 256
BENCH_INFO_SEED = 1000     # information words of rank 0
BENCH_NOISE_SEED = 17      # first of the benchmark's LLR buffers
EARLY_NOISE_SEED = 31      # first buffer of its early-exit context runs


@pytest.fixture(scope="module")
def ldpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01567_gb300 import build
    build.build()
    from paper_1609_01567_gb300 import ldpc as mod
    return mod


@pytest.fixture(scope="module")
def code():
    return I.large_code_n64800()


def threads():
    return max(1, os.cpu_count() or 1)


def philox_llr(oracle_mod, code, frames, ebn0, noise_seed):
    cw = I.encode_ira(code, I.random_info(frames, code.k, seed=BENCH_INFO_SEED))
    lam = oracle_mod.gen_awgn(noise_seed, 0, frames, code.n, I.sigma2_from_ebn0(ebn0, code.rate), cw)
    return cw, lam.astype(np.float32)


def to_host(out):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def exact_except_near_zero(got, ref, frames):
    same = (got["bits"] == ref["bits"]).all(axis=1) & (got["iters"] == ref["iters"]) & (got["ok"] == ref["ok"])
    exempt = near_zero_frames(ref["post"])
    bad = np.flatnonzero(~same & ~exempt)
    detail = [(int(frames[f]), int(got["iters"][f]), int(ref["iters"][f]), int(got["ok"][f]), int(ref["ok"][f]),
               int((got["bits"][f] != ref["bits"][f]).sum())) for f in bad[:10]]
    return bad, exempt, detail


def test_benchmark_launch_every_frame_matches_oracle(ldpc, oracle_mod, code):
    """All 256 frames of the timed call (max_iter 10 fixed, no posteriors,
    default streams and frames per lane): bits, iterations and flags equal the
    oracle's; the same call with posteriors is within tolerance on every
    frame; the profiled form the benchmark times gives the same results."""
    cw, llr = philox_llr(oracle_mod, code, BENCH_FRAMES, 1.0, BENCH_NOISE_SEED)
    h = ldpc.code_from_inputs(code)
    dev = torch.from_numpy(llr).cuda()
    kw = dict(early_exit=False, msg_dtype="f32", streams=0, frames_per_lane=0)
    got = to_host(ldpc.ldpc_decode(h, dev, 10, want_post=False, **kw))
    timed = to_host(ldpc.ldpc_decode(h, dev, 10, want_post=False, profile=2, **kw))
    ldpc.ldpc_prof_read(h, reset=True)
    for k in ("bits", "iters", "ok"):
        np.testing.assert_array_equal(timed[k], got[k], err_msg=f"profiled call {k}")
    ref = oracle_mod.decode(code, llr.astype(np.float64), 10, early_exit=False, n_threads=threads())
    bad, exempt, detail = exact_except_near_zero(got, ref, np.arange(BENCH_FRAMES))
    assert bad.size == 0, f"frames off the oracle (f, it_gpu, it_orc, ok_gpu, ok_orc, dbits): {detail}"
    post = to_host(ldpc.ldpc_decode(h, dev, 10, want_post=True, **kw))
    for k in ("bits", "iters", "ok"):
        np.testing.assert_array_equal(post[k], got[k], err_msg=f"with posteriors {k}")
    ok = close(post["post"], ref["post"]).all(axis=1)
    worst = float(np.abs(post["post"] - ref["post"]).max())
    assert np.all(ok | exempt), (np.flatnonzero(~ok & ~exempt)[:10], worst)
    assert (got["iters"] == 10).all()
    print(f"n64800 benchmark launch: {BENCH_FRAMES} frames, {int(exempt.sum())} exempt, "
          f"{int((ref['ok'] == 1).sum())} codewords after 10 iterations, worst |dpost| {worst:.2e}")


@pytest.mark.parametrize("ebn0", [1.2, 1.6])
def test_early_exit_max_iter_50_matches_oracle(ldpc, oracle_mod, code, ebn0):
    """max_iter 50 with per-frame early exit on 512 frames (two stream halves
    of two 128-frame groups each): 32 frames spread over all four groups
    against the oracle. Bits, iterations and flags exact (near-zero frames
    logged); posteriors within tolerance on the frames that stop within 20
    iterations (longer trajectories carry FP32 rounding over more passes and
    are covered by the lock-step tests)."""
    F = 512
    cw, llr = philox_llr(oracle_mod, code, F, ebn0, EARLY_NOISE_SEED)
    h = ldpc.code_from_inputs(code)
    got = to_host(ldpc.ldpc_decode(h, torch.from_numpy(llr).cuda(), 50, early_exit=True, want_post=True))
    sample = np.unique(np.concatenate([np.linspace(0, F - 1, 28).astype(int), [127, 128, 255, 256]]))
    assert sample.size >= 32 and all(((sample // 128) == g).any() for g in range(4))
    ref = oracle_mod.decode(code, llr[sample].astype(np.float64), 50, early_exit=True, n_threads=threads())
    sub = {k: v[sample] for k, v in got.items()}
    bad, exempt, detail = exact_except_near_zero(sub, ref, sample)
    assert bad.size == 0, f"frames off the oracle (f, it_gpu, it_orc, ok_gpu, ok_orc, dbits): {detail}"
    short = ref["iters"] <= 20
    okp = close(sub["post"], ref["post"]).all(axis=1)
    assert np.all(okp | exempt | ~short), sample[~okp & ~exempt & short]
    drift = float(np.abs(sub["post"] - ref["post"])[~short].max()) if (~short).any() else 0.0
    assert (ref["ok"] == 1).mean() > 0.9
    print(f"n64800 early exit {ebn0} dB: {sample.size} frames, iterations {int(ref['iters'].min())}-"
          f"{int(ref['iters'].max())} (mean {ref['iters'].mean():.1f}), {int(exempt.sum())} exempt, "
          f"worst |dpost| beyond 20 iterations {drift:.2e}")


@pytest.mark.parametrize("msg", ["f32", "bf16"])
def test_early_exit_narrow_tail_is_bit_exact(ldpc, oracle_mod, code, msg):
    """The early-exit form on the benchmark's 256 frames at 1.6 dB: after
    about 20 passes at most 64 frames are still decoding, and from the next
    compaction on the library runs them as one 64-frame group at two frames
    per lane (the narrow tail, picked on the device). That decode equals,
    bit for bit, the one-stream decode and the two-frames-per-lane decode
    (neither has a narrow tail; the second compacts 64-frame groups
    throughout): bits, iterations, flags and posteriors."""
    F = BENCH_FRAMES
    _, llr = philox_llr(oracle_mod, code, F, 1.6, EARLY_NOISE_SEED)
    h = ldpc.code_from_inputs(code)
    dev = torch.from_numpy(llr).cuda()
    got = to_host(ldpc.ldpc_decode(h, dev, 50, early_exit=True, want_post=True, msg_dtype=msg))
    late = int((got["iters"] > 21).sum())
    assert 1 <= late <= 64, late  # the tail runs narrow after the compaction at pass 21
    one = to_host(ldpc.ldpc_decode(h, dev, 50, early_exit=True, want_post=True, msg_dtype=msg, streams=1))
    two = to_host(ldpc.ldpc_decode(h, dev, 50, early_exit=True, want_post=True, msg_dtype=msg, frames_per_lane=2))
    for other, name in ((one, "one stream"), (two, "two frames per lane")):
        for k in ("bits", "iters", "ok", "post"):
            np.testing.assert_array_equal(other[k], got[k], err_msg=f"{name} {k}")
    print(f"n64800 1.6 dB {msg}: {late} frames beyond 21 iterations, iterations up to {int(got['iters'].max())}")


def test_uneven_stream_split_is_bit_exact(ldpc, oracle_mod, code):
    """Padded frame counts that are an odd number of frame groups split
    unevenly over the two pass streams: 300 frames (three 128-frame groups,
    256 + 128 by default) and 165 frames at two per lane (three 64-frame
    groups, 128 + 64 with streams=2). The early-exit decode, whose
    compaction runs across the split, and a fixed-iteration decode each equal
    the one-stream decode bit for bit."""
    _, llr = philox_llr(oracle_mod, code, 300, 1.4, EARLY_NOISE_SEED)
    h = ldpc.code_from_inputs(code)
    for F, kw in ((300, {}), (165, {"frames_per_lane": 2, "streams": 2})):
        dev = torch.from_numpy(llr[:F]).cuda()
        for max_iter, early in ((30, True), (5, False)):
            two = to_host(ldpc.ldpc_decode(h, dev, max_iter, early_exit=early, want_post=True, **kw))
            one = to_host(ldpc.ldpc_decode(h, dev, max_iter, early_exit=early, want_post=True, streams=1,
                                           frames_per_lane=kw.get("frames_per_lane", 0)))
            for k in ("bits", "iters", "ok", "post"):
                np.testing.assert_array_equal(two[k], one[k], err_msg=f"{F} frames, max_iter {max_iter} {k}")
