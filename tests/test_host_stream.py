"""Streaming decode of host batches (copies overlapping decodes) returns what
per-batch device decodes return."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("n_batches,frames", [(1, 64), (2, 33), (5, 100)])
def test_stream_equals_device_decodes(ldpc, n_batches, frames):
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    s2 = I.sigma2_from_ebn0(1.75, code.rate)
    llrs = [torch.from_numpy(I.gaussian_llr(np.zeros((frames, code.n), np.uint8), s2, seed=b)).pin_memory()
            for b in range(n_batches)]
    outs = ldpc.ldpc_decode_host_stream(h, llrs, 20, early_exit=True)
    for b in range(n_batches):
        ref = ldpc.ldpc_decode(h, llrs[b].cuda(), 20, early_exit=True, want_post=False)
        torch.cuda.synchronize()
        for k in ("bits", "iters", "ok"):
            np.testing.assert_array_equal(outs[b][k].numpy(), ref[k].cpu().numpy(), err_msg=f"batch {b} {k}")


def test_stream_shared_outputs_hold_the_last_batch(ldpc):
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    s2 = I.sigma2_from_ebn0(1.5, code.rate)
    llrs = [torch.from_numpy(I.gaussian_llr(np.zeros((40, code.n), np.uint8), s2, seed=50 + b)) for b in range(4)]
    shared = {"bits": torch.empty((40, code.n), dtype=torch.uint8), "iters": torch.empty(40, dtype=torch.int32),
              "ok": torch.empty(40, dtype=torch.uint8)}
    ldpc.ldpc_decode_host_stream(h, llrs, 10, early_exit=False, outs=[shared] * 4, rule="min_sum", rule_alpha=0.8)
    ref = ldpc.ldpc_decode(h, llrs[-1].cuda(), 10, early_exit=False, want_post=False, rule="min_sum", rule_alpha=0.8)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(shared["bits"].numpy(), ref["bits"].cpu().numpy())
    np.testing.assert_array_equal(shared["iters"].numpy(), ref["iters"].cpu().numpy())
    assert ldpc.ldpc_decode_host_stream(h, [], 10) == []


@pytest.mark.parametrize("msg", ["f32", "bf16"])
def test_stream_at_the_benchmark_configuration(ldpc, msg):
    """The end-to-end configuration of the benchmark: n = 64800, 256 frames,
    10 fixed iterations, six batches through the two staging slots (each
    slot's decode captured as a graph and replayed), and the one-call host
    entry point; every batch equals the device decode bit for bit."""
    code = I.large_code_n64800()
    h = ldpc.code_from_inputs(code)
    s2 = I.sigma2_from_ebn0(1.0, code.rate)
    llrs = [ldpc.ldpc_gen_awgn(70 + b, 0, 256, code.n, s2).cpu().pin_memory() for b in range(3)]
    batches = [llrs[b % 3] for b in range(6)]
    outs = ldpc.ldpc_decode_host_stream(h, batches, 10, early_exit=False, msg_dtype=msg)
    refs = []
    for b in range(3):
        ref = ldpc.ldpc_decode(h, llrs[b].cuda(), 10, early_exit=False, want_post=False, msg_dtype=msg)
        torch.cuda.synchronize()
        refs.append({k: v.cpu().numpy() for k, v in ref.items()})
    for b in range(6):
        for k in ("bits", "iters", "ok"):
            np.testing.assert_array_equal(outs[b][k].numpy(), refs[b % 3][k], err_msg=f"batch {b} {k}")
    one = ldpc.ldpc_decode_host(h, llrs[1], 10, early_exit=False, msg_dtype=msg)
    for k in ("bits", "iters", "ok"):
        np.testing.assert_array_equal(one[k].numpy(), refs[1][k], err_msg=f"one call {k}")


def test_one_call_in_two_parts(ldpc):
    """A large one-call host decode runs as two parts whose copies overlap
    the other part's decode (here 300 frames: 256 + 44, and 256: 128 + 128),
    with early exit and posteriors; repeated calls replay captured graphs.
    Every call equals the device decode of the whole batch bit for bit."""
    code = I.large_code_n64800()
    h = ldpc.code_from_inputs(code)
    s2 = I.sigma2_from_ebn0(1.4, code.rate)
    for F in (300, 256):
        llr = ldpc.ldpc_gen_awgn(90 + F, 0, F, code.n, s2).cpu().pin_memory()
        ref = ldpc.ldpc_decode(h, llr.cuda(), 30, want_post=True)
        torch.cuda.synchronize()
        ref = {k: v.cpu().numpy() for k, v in ref.items()}
        for rep in range(3):
            got = ldpc.ldpc_decode_host(h, llr, 30, want_post=True)
            for k in ("bits", "iters", "ok", "post"):
                np.testing.assert_array_equal(np.asarray(got[k]), ref[k], err_msg=f"{F} frames, call {rep}, {k}")
