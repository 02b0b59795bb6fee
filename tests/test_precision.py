"""Reduced-precision messages (FP16 / BF16 storage, FP32 node sums) vs the
FP64 oracle and vs FP32 messages, in frame error rate.

Both sides draw the channel from the same counter-based generator (each its
own implementation), so they see the same noise up to float rounding; the
comparison is statistical: 95% Wilson intervals must overlap.
"""
import os

import numpy as np
import pytest

from paper_1609_01567_gb300 import ber
from paper_1609_01567_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ldpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01567_gb300 import build
    build.build()
    from paper_1609_01567_gb300 import ldpc as mod
    return mod


def overlap(a, b):
    return a[0] <= b[1] and b[0] <= a[1]


def test_count_errors_kernel(ldpc):
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2, size=(50, 333), dtype=np.uint8)
    ref = rng.integers(0, 2, size=(50, 333), dtype=np.uint8)
    ref[:10] = bits[:10]
    iters = rng.integers(0, 9, size=50).astype(np.int32)
    ok = rng.integers(0, 2, size=50).astype(np.uint8)
    c = ldpc.ldpc_count_errors(torch.from_numpy(bits).cuda(), torch.from_numpy(ref).cuda(),
                               torch.from_numpy(iters).cuda(), torch.from_numpy(ok).cuda()).cpu().numpy()
    assert c[0] == (bits != ref).sum() and c[1] == (bits != ref).any(axis=1).sum()
    assert c[2] == iters.sum() and c[3] == (ok == 0).sum()
    z = ldpc.ldpc_count_errors(torch.from_numpy(bits).cuda()).cpu().numpy()
    assert z[0] == bits.sum() and z[1] == bits.any(axis=1).sum()


def test_fer_of_message_precisions_against_oracle_n1008(ldpc, oracle_mod):
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    frames, ebn0, seed = 3000, 1.5, 9
    s2 = I.sigma2_from_ebn0(ebn0, code.rate)
    lam = oracle_mod.gen_awgn(seed, 0, frames, code.n, s2)
    ref = oracle_mod.decode(code, lam, 50, want_post=False, n_threads=os.cpu_count())
    k_ref = int(ref["bits"].any(axis=1).sum())
    ci_ref = ber.wilson(k_ref, frames)
    assert 30 < k_ref < frames - 30
    for msg in ("f32", "f16", "bf16"):
        c = ber.simulate(h, code, ebn0, frames, batch=512, max_iter=50, msg_dtype=msg, seed=seed)
        ci = ber.wilson(c.frame_errors, c.frames)
        assert overlap(ci, ci_ref), (msg, c.frame_errors, k_ref)
        if msg == "f32":
            # same noise up to float rounding: the FP32 decoder fails on
            # nearly the same frames as the oracle
            assert abs(c.frame_errors - k_ref) <= max(3, k_ref // 50), (c.frame_errors, k_ref)


def test_fer_of_message_precisions_n64800(ldpc):
    code = I.large_code_n64800()
    h = ldpc.code_from_inputs(code)
    res = {}
    for msg in ("f32", "f16", "bf16"):
        c = ber.simulate(h, code, 1.0, 2048, batch=1024, max_iter=50, msg_dtype=msg, seed=4)
        res[msg] = c
    k32 = res["f32"].frame_errors
    assert 20 < k32 < 2048 - 20
    for msg in ("f16", "bf16"):
        assert overlap(ber.wilson(res[msg].frame_errors, 2048), ber.wilson(k32, 2048)), (msg, res[msg], k32)
