"""The decode server: each request's results are the same alone and in the
mix of concurrent requests, and equal the plain decoder's."""
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
    from paper_1609_01567_gb300 import mixed as M
    codes = I.mixed_codes()[:6]
    handles = [ldpc.code_from_inputs(c) for c in codes]
    rng = np.random.default_rng(5)
    reqs = []
    for r in range(40):
        ci = int(rng.integers(0, len(codes)))
        f = int(rng.integers(1, 65))
        c = codes[ci]
        cw = torch.from_numpy(I.encode_ira(c, I.random_info(f, c.k, seed=1000 + r))).cuda()
        s2 = I.sigma2_from_ebn0(M.EBN0_AT_FER_1E2[c.name], c.rate)
        reqs.append((ci, ldpc.ldpc_gen_awgn(500 + r, 0, f, c.n, s2, cw)))
    return codes, handles, reqs


def host(o):
    return {k: v.cpu().numpy() for k, v in o.items()}


@pytest.mark.parametrize("msg,rule", [("f32", "sum_product"), ("f16", "sum_product"), ("i8", "sum_product"),
                                      ("f32", "min_sum")])
def test_same_result_alone_and_in_the_mix(ldpc, setup, msg, rule):
    codes, handles, reqs = setup
    kw = dict(rule=rule, rule_alpha=0.8) if rule == "min_sum" else {}
    srv = ldpc.ldpc_server_create(handles, max_batch_frames=256, max_slots=3, msg_dtype=msg, max_iter=30, **kw)
    alone = []
    for ci, llr in reqs:  # one request at a time
        rid, o = ldpc.ldpc_server_submit(srv, ci, llr, want_post=True)
        ldpc.ldpc_server_wait(srv, rid, timeout_ms=60000)
        alone.append(host(o))
    subs = [ldpc.ldpc_server_submit(srv, ci, llr, want_post=True) for ci, llr in reqs]  # all at once
    lat = [ldpc.ldpc_server_wait(srv, rid, timeout_ms=60000) for rid, _ in subs]
    stats = ldpc.ldpc_server_stats(srv)
    srv.close()
    assert stats["completed"] == 2 * len(reqs) and stats["batches"] < 2 * len(reqs)  # the mix was batched
    assert all(x >= 0.0 for x in lat)
    for (rid, o), a, (ci, llr) in zip(subs, alone, reqs):
        got = host(o)
        for k in ("bits", "iters", "ok", "post"):
            np.testing.assert_array_equal(got[k], a[k], err_msg=f"code {ci} {k}")
        if msg == "f32":
            ref = host(ldpc.ldpc_decode(handles[ci], llr, 30, msg_dtype=msg, streams=1, **kw))
            for k in ("bits", "iters", "ok", "post"):
                np.testing.assert_array_equal(got[k], ref[k])


def test_backpressure_and_errors(ldpc, setup):
    codes, handles, reqs = setup
    srv = ldpc.ldpc_server_create(handles, max_batch_frames=128, max_slots=1, max_pending_frames=16)
    ci, llr = next((c, l) for c, l in reqs if l.shape[0] > 16)
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_server_submit(srv, ci, llr)
    assert e.value.status == -6
    import ctypes
    rid = ctypes.c_uint64()
    buf = torch.empty(llr.shape, dtype=torch.uint8, device="cuda")
    st = ldpc.library().ldpc_server_submit(srv.handle, len(handles), ctypes.c_void_p(llr.data_ptr()), llr.shape[0],
                                          ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                          ctypes.c_void_p(buf.data_ptr()), None, ctypes.byref(rid))
    assert st == -1
    rid, o = ldpc.ldpc_server_submit(srv, reqs[0][0], reqs[0][1][:8])
    ldpc.ldpc_server_wait(srv, rid, timeout_ms=60000)
    srv.close()
