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


def static_call(ldpc, h, llr_dev, max_iter, early_exit):
    """Call ldpc_decode_static through the C ABI with preallocated outputs."""
    lib = ldpc.library()
    f, n = llr_dev.shape
    bits = torch.empty((f, n), dtype=torch.uint8, device=llr_dev.device)
    iters = torch.empty((f,), dtype=torch.int32, device=llr_dev.device)
    ok = torch.empty((f,), dtype=torch.uint8, device=llr_dev.device)
    post = torch.empty((f, n), dtype=torch.float32, device=llr_dev.device)
    opts = ldpc.ldpc_decode_opts_t(early_exit=1 if early_exit else 0, l_max=20.0, msg_dtype=0)
    vp = ctypes.c_void_p
    st = lib.ldpc_decode_static(h.handle, vp(llr_dev.data_ptr()), f, max_iter, ctypes.byref(opts), vp(bits.data_ptr()),
                                vp(iters.data_ptr()), vp(ok.data_ptr()), vp(post.data_ptr()),
                                vp(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.ldpc_last_error().decode()
    torch.cuda.synchronize()
    return {"bits": bits.cpu().numpy(), "iters": iters.cpu().numpy(), "ok": ok.cpu().numpy(),
            "post": post.cpu().numpy()}


def test_static_scratch_decode_matches_ldpc_decode(ldpc):
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    cw = I.encode_ira(code, I.random_info(600, code.k, seed=77))
    llr = I.gaussian_llr(cw, I.sigma2_from_ebn0(1.75, code.rate), seed=78)
    # two calls in a row with different batches and settings: the second must
    # not see anything the first left in the shared scratch
    for sub, max_iter, early in ((slice(0, 300), 30, True), (slice(300, 600), 12, False)):
        llr_dev = torch.from_numpy(np.ascontiguousarray(llr[sub])).cuda()
        got = static_call(ldpc, h, llr_dev, max_iter, early)
        ref = ldpc.ldpc_decode(h, llr_dev, max_iter, early_exit=early)
        torch.cuda.synchronize()
        ref = {k: v.cpu().numpy() for k, v in ref.items()}
        np.testing.assert_array_equal(got["bits"], ref["bits"])
        np.testing.assert_array_equal(got["iters"], ref["iters"])
        np.testing.assert_array_equal(got["ok"], ref["ok"])
        assert close(got["post"], ref["post"]).all()


def test_static_scratch_rejects_oversized_batches(ldpc):
    code = I.large_code_n64800()
    h = ldpc.code_from_inputs(code)
    llr_dev = torch.zeros((256, code.n), dtype=torch.float32, device="cuda")
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_decode_static(h, llr_dev, 10)
    assert e.value.status == -1 and "static scratch holds" in str(e.value)
