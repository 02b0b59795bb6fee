"""The allocation-free decode entry point against the regular one.

ldpc_decode_static serves callers that may not allocate device memory when
they decode (a receive chain that must not stall on cudaMalloc's device-wide
synchronisation, or a plug-in limited to another framework's memory pool):
it keeps its scratch in a fixed 64 MiB device array instead. Its results must
equal ldpc_decode's on the same inputs, call after call, although every call
reuses (and must correctly clear) the same scratch. This file is collected
last, so a run that stops at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1609_01567_gb300 import inputs as I
from tests.parity import close

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


def static_call(ldpc, h, llr_dev, max_iter, early_exit, out=None, **kw):
    """Call ldpc_decode_static through the C ABI; outputs are preallocated
    here unless given in ``out`` (then the call allocates nothing at all)."""
    lib = ldpc.library()
    f, n = llr_dev.shape
    if out is None:
        out = {"bits": torch.empty((f, n), dtype=torch.uint8, device=llr_dev.device),
               "iters": torch.empty((f,), dtype=torch.int32, device=llr_dev.device),
               "ok": torch.empty((f,), dtype=torch.uint8, device=llr_dev.device),
               "post": torch.empty((f, n), dtype=torch.float32, device=llr_dev.device)}
    opts = ldpc._opts(early_exit, 20.0, kw.pop("msg_dtype", "f32"), False, None, **kw)
    vp = ctypes.c_void_p
    st = lib.ldpc_decode_static(h.handle, vp(llr_dev.data_ptr()), f, max_iter, ctypes.byref(opts),
                                vp(out["bits"].data_ptr()), vp(out["iters"].data_ptr()), vp(out["ok"].data_ptr()),
                                vp(out["post"].data_ptr()), vp(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.ldpc_last_error().decode()
    return out


def host(out):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def assert_same_decode(got, ref, what):
    np.testing.assert_array_equal(got["bits"], ref["bits"], err_msg=what)
    np.testing.assert_array_equal(got["iters"], ref["iters"], err_msg=what)
    np.testing.assert_array_equal(got["ok"], ref["ok"], err_msg=what)
    assert close(got["post"], ref["post"]).all(), what


def test_static_scratch_decode_matches_ldpc_decode(ldpc):
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    cw = I.encode_ira(code, I.random_info(600, code.k, seed=77))
    llr = I.gaussian_llr(cw, I.sigma2_from_ebn0(1.75, code.rate), seed=78)
    # two calls in a row with different batches and settings: the second must
    # not see anything the first left in the shared scratch
    for sub, max_iter, early in ((slice(0, 300), 30, True), (slice(300, 600), 12, False)):
        llr_dev = torch.from_numpy(np.ascontiguousarray(llr[sub])).cuda()
        got = host(static_call(ldpc, h, llr_dev, max_iter, early))
        ref = host(ldpc.ldpc_decode(h, llr_dev, max_iter, early_exit=early))
        assert_same_decode(got, ref, f"{sub} max_iter={max_iter} early_exit={early}")


def test_static_scratch_reuse_across_layouts(ldpc):
    """Calls that carve the shared array differently, one after the other:
    each places its messages, posteriors, LLRs and flag rows at other offsets
    than the call before, over what that call left there. A large early-exit
    FP16 decode (2048 padded frames), then a small FP32 decode of another
    code, then int8 messages with offset min-sum, then eight frames per lane
    with BF16 messages; every one equals ldpc_decode with the same options."""
    c1008, c576 = I.small_code_n1008(), I.mixed_code(0)
    h1008, h576 = ldpc.code_from_inputs(c1008), ldpc.code_from_inputs(c576)
    calls = [
        (c1008, h1008, 2000, 1.5, 40, True, dict(msg_dtype="f16")),
        (c576, h576, 37, 3.5, 25, True, dict()),
        (c1008, h1008, 500, 2.0, 30, True, dict(msg_dtype="i8", rule="min_sum", rule_alpha=0.9, rule_beta=0.15)),
        (c1008, h1008, 300, 1.75, 18, False, dict(msg_dtype="bf16", frames_per_lane=8)),
        (c576, h576, 1, 3.0, 10, True, dict()),
    ]
    for i, (code, h, f, ebn0, max_iter, early, kw) in enumerate(calls):
        llr = I.gaussian_llr(np.zeros((f, code.n), np.uint8), I.sigma2_from_ebn0(ebn0, code.rate), seed=300 + i)
        llr_dev = torch.from_numpy(llr).cuda()
        got = host(static_call(ldpc, h, llr_dev, max_iter, early, **dict(kw)))
        ref = host(ldpc.ldpc_decode(h, llr_dev, max_iter, early_exit=early, **kw))
        assert_same_decode(got, ref, f"call {i}: {code.name} F={f} {kw}")
        if i == 0:
            assert (got["iters"] < max_iter).mean() > 0.5  # early exit retired most frames


def test_static_call_allocates_no_device_memory(ldpc):
    """The property the entry point exists for: with the code made and the
    outputs provided by the caller, a call changes neither the device's free
    memory nor PyTorch's allocation (one identical call first, so that lazily
    loaded kernels are already resident)."""
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    llr = I.gaussian_llr(np.zeros((200, code.n), np.uint8), I.sigma2_from_ebn0(2.0, code.rate), seed=5)
    llr_dev = torch.from_numpy(llr).cuda()
    out = {"bits": torch.empty((200, code.n), dtype=torch.uint8, device="cuda"),
           "iters": torch.empty((200,), dtype=torch.int32, device="cuda"),
           "ok": torch.empty((200,), dtype=torch.uint8, device="cuda"),
           "post": torch.empty((200, code.n), dtype=torch.float32, device="cuda")}
    static_call(ldpc, h, llr_dev, 20, True, out=out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        static_call(ldpc, h, llr_dev, 20, True, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0, (free0, free1)


def test_static_scratch_rejects_oversized_batches(ldpc):
    code = I.large_code_n64800()
    h = ldpc.code_from_inputs(code)
    llr_dev = torch.zeros((256, code.n), dtype=torch.float32, device="cuda")
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_decode_static(h, llr_dev, 10)
    assert e.value.status == -1 and "static scratch holds" in str(e.value)
