"""Mixed-code batches (one CUDA graph over several codes) against per-code
decodes and against the oracle on the unbounded-degree code."""
import numpy as np
import pytest

from paper_1609_01567_gb300 import inputs as I
from tests.parity import compare_decodes

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
def mixed(ldpc):
    from paper_1609_01567_gb300 import mixed as M
    codes = I.mixed_codes()
    frames = [max(1, f // 8) for f in I.zipf_frames(4096, len(codes))]  # a lighter copy of the workload
    handles = [ldpc.code_from_inputs(c) for c in codes]
    llrs, sent = M.make_llrs(codes, frames)
    return codes, frames, handles, llrs, sent


def host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_batch_graph_equals_per_code_decodes(ldpc, mixed):
    codes, frames, handles, llrs, sent = mixed
    refs = [host(ldpc.ldpc_decode(h, l, 50)) for h, l in zip(handles, llrs)]
    b = ldpc.ldpc_batch_create(handles, frames, 50)
    outs = ldpc.ldpc_batch_run(b, llrs, want_post=True)  # direct launches
    first = [host(o) for o in outs]
    for rep in range(3):  # graph capture, then replays
        outs = ldpc.ldpc_batch_run(b, llrs, outs)
        torch.cuda.synchronize()
        for i, (o, ref) in enumerate(zip(outs, refs)):
            got = host(o)
            for k in ("bits", "iters", "ok", "post"):
                np.testing.assert_array_equal(got[k], ref[k], err_msg=f"item {i} rep {rep} {k}")
                np.testing.assert_array_equal(first[i][k], ref[k])
    assert ldpc.ldpc_batch_info(b, 0)["kernels_per_run"] > 0
    b.close()


def test_batch_tuning_keeps_results(ldpc, mixed):
    codes, frames, handles, llrs, sent = mixed
    refs = [host(ldpc.ldpc_decode(h, l, 50, want_post=False)) for h, l in zip(handles, llrs)]
    for msg in ("f32", "bf16"):
        b = ldpc.ldpc_batch_create(handles, frames, 50, msg_dtype=msg)
        ldpc.ldpc_batch_tune(b, llrs)
        for i in range(len(codes)):
            info = ldpc.ldpc_batch_info(b, i)
            assert info["frames_per_lane"] in (1, 2, 4, 8) and info["check_schedule"] in (1, 2)
        outs = ldpc.ldpc_batch_run(b, llrs)
        outs = ldpc.ldpc_batch_run(b, llrs, outs)
        torch.cuda.synchronize()
        for i, (o, ref) in enumerate(zip(outs, refs)):
            got = host(o)
            if msg == "f32":
                for k in ("bits", "iters", "ok"):
                    np.testing.assert_array_equal(got[k], ref[k], err_msg=f"item {i} {k}")
            else:  # reduced precision: same frames succeed up to a few
                assert abs(int(got["ok"].sum()) - int(ref["ok"].sum())) <= max(2, frames[i] // 50)
        b.close()


def test_unbounded_degree_code_matches_oracle(ldpc, oracle_mod):
    code = I.mixed_codes()[4]  # degree-64 variable, degree-96 check
    h = ldpc.code_from_inputs(code)
    cw = I.encode_ira(code, I.random_info(40, code.k, seed=3))
    llr = I.gaussian_llr(cw, I.sigma2_from_ebn0(3.0, code.rate), seed=4)
    got = host(ldpc.ldpc_decode(h, torch.from_numpy(llr).cuda(), 12, early_exit=False))
    ref = oracle_mod.decode(code, llr.astype(np.float64), 12, early_exit=False, n_threads=8)
    bad, exempt = compare_decodes(got, ref)
    assert bad.size == 0, bad


@pytest.mark.parametrize("msg,rule", [("i8", "sum_product"), ("f32", "sp_table"), ("bf16", "min_sum"),
                                      ("f32", "min_sum_adaptive")])
def test_batch_other_formats_and_rules(ldpc, mixed, msg, rule):
    """The graph batch gives per-code decodes' results for every message
    format and check rule (the adaptive rule with each code's own table)."""
    codes, frames, handles, llrs, sent = mixed
    kw = dict(rule=rule, rule_alpha=0.8) if rule == "min_sum" else dict(rule=rule)
    if rule == "min_sum_adaptive":
        for i, h in enumerate(handles):
            ldpc.ldpc_code_set_rule_table(h, [0.9 - 0.02 * ((d + i) % 7) for d in range(100)], [0.05 * (d % 3) for d in range(100)])
    refs = [host(ldpc.ldpc_decode(h, l, 30, want_post=False, msg_dtype=msg, **kw)) for h, l in zip(handles, llrs)]
    b = ldpc.ldpc_batch_create(handles, frames, 30, msg_dtype=msg, **kw)
    outs = ldpc.ldpc_batch_run(b, llrs)
    outs = ldpc.ldpc_batch_run(b, llrs, outs)  # captured graph
    torch.cuda.synchronize()
    for i, (o, ref) in enumerate(zip(outs, refs)):
        got = host(o)
        for k in ("bits", "iters", "ok"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"item {i} {msg} {rule} {k}")
    b.close()
