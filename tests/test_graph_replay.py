"""Graph replay of repeated decodes: a decode whose shape, options and
buffers recur is captured into a CUDA graph and replayed. Replays must read
the buffers' current contents and give exactly what a direct decode gives
(profiled decodes always run directly)."""
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


def llrs(code, F, ebn0, seed):
    return torch.from_numpy(I.gaussian_llr(np.zeros((F, code.n), np.uint8), I.sigma2_from_ebn0(ebn0, code.rate),
                                           seed=seed)).cuda()


def direct(ldpc, h, llr, max_iter, **kw):
    out = ldpc.ldpc_decode(h, llr, max_iter, profile=True, **kw)
    torch.cuda.synchronize()
    ldpc.ldpc_prof_read(h, reset=True)
    return {k: v.cpu().numpy() for k, v in out.items()}


def same(a, b):
    for k in a:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


@pytest.mark.parametrize("kw", [dict(), dict(msg_dtype="bf16", early_exit=False), dict(rule="min_sum", rule_alpha=0.8),
                                dict(streams=1, frames_per_lane=2)])
def test_replays_follow_buffer_contents(ldpc, kw):
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    buf = llrs(code, 300, 1.5, seed=1)
    out = None
    for rnd in range(4):  # direct, captured, replayed, replayed
        buf.copy_(llrs(code, 300, 1.5, seed=10 + rnd))
        out = ldpc.ldpc_decode(h, buf, 25, out=out, **kw)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        same(got, direct(ldpc, h, buf, 25, **kw))


def test_alternating_buffers_and_workspace_growth(ldpc):
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    a, b = llrs(code, 64, 2.0, seed=3), llrs(code, 64, 2.0, seed=4)
    oa = ob = None
    for _ in range(3):
        oa = ldpc.ldpc_decode(h, a, 20, out=oa)
        ob = ldpc.ldpc_decode(h, b, 20, out=ob)
    torch.cuda.synchronize()
    same({k: v.cpu().numpy() for k, v in oa.items()}, direct(ldpc, h, a, 20))
    same({k: v.cpu().numpy() for k, v in ob.items()}, direct(ldpc, h, b, 20))
    big = llrs(code, 9000, 2.0, seed=5)  # more than one chunk; grows the workspace
    for _ in range(3):
        ob2 = ldpc.ldpc_decode(h, big, 6)
    torch.cuda.synchronize()
    same({k: v.cpu().numpy() for k, v in ob2.items()}, direct(ldpc, h, big, 6))
    for _ in range(3):
        oa = ldpc.ldpc_decode(h, a, 20, out=oa)
    torch.cuda.synchronize()
    same({k: v.cpu().numpy() for k, v in oa.items()}, direct(ldpc, h, a, 20))


def test_host_entry_replays_and_counts_kernels(ldpc):
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    host = llrs(code, 100, 1.75, seed=6).cpu().pin_memory()
    ref = direct(ldpc, h, host.cuda(), 15)
    ldpc.ldpc_prof_read(h, reset=True)
    for _ in range(3):
        got = ldpc.ldpc_decode_host(h, host, 15)
        for k in ("bits", "iters", "ok"):
            np.testing.assert_array_equal(np.asarray(got[k]), ref[k], err_msg=k)
    # replayed graphs still count their kernels
    k3 = ldpc.ldpc_prof_read(h, reset=True)["kernels"]
    ldpc.ldpc_decode_host(h, host, 15)
    k1 = ldpc.ldpc_prof_read(h, reset=True)["kernels"]
    assert k1 > 0 and k3 == 3 * k1


def test_replays_read_the_current_rule_table(ldpc):
    """A captured decode reads the code's degree table at replay time, so a
    new table shows in the next replay."""
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    buf = llrs(code, 300, 1.5, seed=21)
    out = None
    for rnd, (a5, a6) in enumerate(((0.7, 0.9), (0.7, 0.9), (0.7, 0.9), (0.95, 0.6), (0.6, 0.8))):
        ldpc.ldpc_code_set_rule_table(h, [1.0] * 5 + [a5, a6], [0.0] * 5 + [0.1, 0.2])
        out = ldpc.ldpc_decode(h, buf, 25, out=out, rule="min_sum_adaptive")
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        same(got, direct(ldpc, h, buf, 25, rule="min_sum_adaptive"))


@pytest.mark.parametrize("code_fn,F", [(I.small_code_n1008, 512), (I.large_code_n64800, 256)])
def test_replays_with_halves_that_stop_far_apart(ldpc, code_fn, F):
    """One half of the batch at high SNR (stops within a few iterations), the
    other near the threshold (runs long), so the two pass streams retire their
    warps at very different passes: replays equal direct decodes bit for bit,
    for max_iter 50 and 23."""
    code = code_fn()
    h = ldpc.code_from_inputs(code)
    lo = {1008: 1.2, 64800: 1.0}[code.n]
    buf = torch.cat([llrs(code, F // 2, 4.0, seed=31), llrs(code, F // 2, lo, seed=32)])
    for max_iter in (50, 23):
        out = None
        for _ in range(4):  # direct, captured, replayed, replayed
            out = ldpc.ldpc_decode(h, buf, max_iter, out=out)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        ref = direct(ldpc, h, buf, max_iter)
        same(got, ref)
        assert ref["iters"][: F // 2].max() < 16 and ref["iters"][F // 2:].max() >= 20, ref["iters"]
