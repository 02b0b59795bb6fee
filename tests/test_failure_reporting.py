"""The bounded-wait give-up path of the pipelined check kernel, driven
without a fault.

The check kernel waits for its row copies with a bounded number of polls; a
warp whose wait runs out sets the call's status word, waits (bounded) for its
own copies still in flight and leaves, and the call then reports iters = -1
and syndrome_ok = 0 for every frame, LDPC_ETIMEOUT from the host-buffer entry
points. A copy that never lands cannot be made without a fault, so the test
hook ldpc_debug_giveup makes one warp take that path after its rows have
landed. The context stays usable: the next decode equals an undisturbed one.
"""
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


@pytest.fixture(scope="module")
def setup(ldpc):
    code = I.small_code_n1008()  # checks of degree 5-6: the pipelined kernel at 256 frames
    h = ldpc.code_from_inputs(code)
    cw = I.encode_ira(code, I.random_info(256, code.k, seed=41))
    llr = I.gaussian_llr(cw, I.sigma2_from_ebn0(2.0, code.rate), seed=42)
    return code, h, llr


def host(out):
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("cta", [0, 5])
def test_given_up_wait_reports_no_results_and_the_next_decode_is_normal(ldpc, setup, cta):
    code, h, llr = setup
    dev = torch.from_numpy(llr).cuda()
    ref = host(ldpc.ldpc_decode(h, dev, 20))
    ldpc.ldpc_debug_giveup(h, cta)
    got = host(ldpc.ldpc_decode(h, dev, 20))
    assert (got["iters"] == -1).all() and (got["ok"] == 0).all()
    # the hook cleared itself; the context and the workspace are intact
    again = host(ldpc.ldpc_decode(h, dev, 20))
    for k in ("bits", "iters", "ok", "post"):
        np.testing.assert_array_equal(again[k], ref[k], err_msg=k)
    assert (ref["iters"] >= 0).all()


def test_host_entry_points_return_etimeout(ldpc, setup):
    code, h, llr = setup
    ldpc.ldpc_debug_giveup(h, 0)
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_decode_host(h, llr, 20)
    assert e.value.status == -5 and "ran out" in str(e.value)
    pinned = [torch.from_numpy(llr).pin_memory() for _ in range(3)]
    ldpc.ldpc_debug_giveup(h, 0)
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_decode_host_stream(h, pinned, 20)
    assert e.value.status == -5
    # unarmed: the same calls succeed and agree with the device entry point
    outs = ldpc.ldpc_decode_host_stream(h, pinned, 20)
    ref = host(ldpc.ldpc_decode(h, torch.from_numpy(llr).cuda(), 20, want_post=False))
    for o in outs:
        np.testing.assert_array_equal(o["bits"].numpy(), ref["bits"])
        np.testing.assert_array_equal(o["iters"].numpy(), ref["iters"])
    ldpc.ldpc_debug_giveup(h, 3)
    ldpc.ldpc_debug_giveup(h, -1)  # disarmed again
    assert (ldpc.ldpc_decode_host(h, llr, 20)["iters"] >= 0).all()
    with pytest.raises(ldpc.LdpcError):
        ldpc.ldpc_debug_giveup(h, -2)
