"""int8 message storage (step 20/127, |k| <= 127) vs the oracle with the same
quantised storage.

The GPU computes each message in FP32 and rounds it to the int8 lattice; the
oracle computes it in FP64 and rounds it the same way. The two stored levels
agree except where the unrounded message lies within FP32 rounding of a
half-step boundary; there they may differ by one level. The lock-step test
checks exactly that, pass by pass, from the GPU's own previous messages.
"""
import numpy as np
import pytest

from paper_1609_01567_gb300 import ber
from paper_1609_01567_gb300 import inputs as I
from tests.parity import close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEP = 20.0 / 127.0
# how close (in steps) the FP64 message must be to a rounding boundary for a
# one-level difference to be accepted: the FP32 path's message error is below
# 1e-4 (the FP32 lock-step tolerance), i.e. 6.4e-4 steps
BOUNDARY = 2e-3


@pytest.fixture(scope="module")
def ldpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_01567_gb300 import build
    build.build()
    from paper_1609_01567_gb300 import ldpc as mod
    return mod


@pytest.fixture(scope="module")
def n1008():
    code = I.small_code_n1008()
    cw = I.encode_ira(code, I.random_info(600, code.k, seed=1200))
    llr = I.gaussian_llr(cw, I.sigma2_from_ebn0(2.0, code.rate), seed=1201)
    return code, cw, llr


def gpu_decode(ldpc, handle, llr, max_iter, **kw):
    out = ldpc.ldpc_decode(handle, torch.from_numpy(np.ascontiguousarray(llr, dtype=np.float32)).cuda(), max_iter,
                           msg_dtype="i8", **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def levels(r):
    k = np.asarray(r, dtype=np.float64) / STEP
    kr = np.round(k)
    assert np.abs(k - kr).max() < 1e-4, "message off the int8 lattice"
    assert np.abs(kr).max() <= 127
    return kr.astype(np.int64)


@pytest.mark.parametrize("rule,alpha,beta", [("sum_product", 1.0, 0.0), ("min_sum", 0.8, 0.2)])
def test_i8_lock_step_passes_n1008(ldpc, oracle_mod, n1008, rule, alpha, beta):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    kw = dict(rule=rule, rule_alpha=alpha, rule_beta=beta)
    orc_rule = "sp" if rule == "sum_product" else "min_sum"
    v_of_edge = oracle_mod.address_iterators(code)["v"]
    lam = llr.astype(np.float64)
    prev_r = None
    n_off = 0
    n_total = 0
    for t in range(0, 41, 4):
        if t > 0:
            prev_r = gpu_decode(ldpc, h, llr, t - 1, early_exit=False, want_r=True, **kw)["r"].astype(np.float64)
        got = gpu_decode(ldpc, h, llr, t, early_exit=False, want_r=True, **kw)
        ref = oracle_mod.sp_pass(code, lam, prev_r, n_threads=8, rule=orc_rule, alpha=alpha, beta=beta, msg="i8")
        raw = oracle_mod.sp_pass(code, lam, prev_r, n_threads=8, rule=orc_rule, alpha=alpha, beta=beta)
        kg, ko = levels(got["r"]), levels(ref["r"])
        off = kg != ko
        # a differing level: one step apart, and the unrounded message sits on
        # a rounding boundary (or on the clamp at 127 levels)
        assert np.abs(kg - ko).max() <= 1, t
        u = np.minimum(np.abs(raw["r"][off]) / STEP, 127.0)
        frac = np.abs(u - np.floor(u) - 0.5)
        assert np.all(frac < BOUNDARY), (t, frac.max())
        n_off += int(off.sum())
        n_total += off.size
        # posteriors: the sum of the stored messages, each differing level
        # moving its bit's posterior by one step
        per_bit = np.zeros_like(got["post"], dtype=np.float64)
        for f in np.flatnonzero(off.any(axis=1)):
            np.add.at(per_bit[f], v_of_edge[off[f]], STEP)
        dpost = np.abs(got["post"].astype(np.float64) - ref["post"])
        assert np.all(dpost <= 1e-4 * np.abs(ref["post"]) + 1e-4 + per_bit + 1e-6), (t, float(dpost.max()))
    assert n_off <= 1e-4 * n_total, (n_off, n_total)
    print(f"int8 lock-step {rule}: {n_off} of {n_total} stored levels one step off (all on boundaries)")


def test_i8_full_decode_n1008(ldpc, oracle_mod, n1008):
    """End to end: nearly every frame decodes to the oracle's bits and
    iteration count; a frame may part ways after a boundary message."""
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    got = gpu_decode(ldpc, h, llr, 50)
    ref = oracle_mod.decode(code, llr.astype(np.float64), 50, n_threads=8, msg="i8")
    same = (got["bits"] == ref["bits"]).all(axis=1) & (got["iters"] == ref["iters"]) & (got["ok"] == ref["ok"])
    assert same.mean() >= 0.97, np.flatnonzero(~same)[:10]
    assert (ref["ok"] == 1).mean() > 0.8
    fe_g = int((got["bits"] != cw).any(axis=1).sum())
    fe_o = int((ref["bits"] != cw).any(axis=1).sum())
    assert abs(fe_g - fe_o) <= max(3, fe_o // 10), (fe_g, fe_o)


def test_i8_schedules_do_not_change_results(ldpc, n1008):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    base = gpu_decode(ldpc, h, llr, 15, frames_per_lane=1, check_schedule=1, streams=1)
    for v, sched, nst, tile in ((2, 1, 1, 0), (4, 2, 1, 0), (4, 2, 2, 0), (8, 2, 2, 0), (2, 2, 2, 64), (0, 0, 0, 0)):
        other = gpu_decode(ldpc, h, llr, 15, frames_per_lane=v, check_schedule=sched, streams=nst, tile_frames=tile)
        for k in ("bits", "iters", "ok", "post"):
            np.testing.assert_array_equal(other[k], base[k], err_msg=f"V={v} schedule={sched} streams={nst} {k}")


def test_i8_fer_against_quantised_oracle_n1008(ldpc, oracle_mod):
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    frames, ebn0, seed = 3000, 1.5, 9
    lam = oracle_mod.gen_awgn(seed, 0, frames, code.n, I.sigma2_from_ebn0(ebn0, code.rate))
    ref = oracle_mod.decode(code, lam, 50, want_post=False, n_threads=16, msg="i8")
    k_ref = int(ref["bits"].any(axis=1).sum())
    c = ber.simulate(h, code, ebn0, frames, batch=512, max_iter=50, msg_dtype="i8", seed=seed)
    assert 30 < k_ref < frames - 30
    assert abs(c.frame_errors - k_ref) <= max(4, k_ref // 20), (c.frame_errors, k_ref)


def test_i8_fer_n64800_close_to_f32(ldpc):
    code = I.large_code_n64800()
    h = ldpc.code_from_inputs(code)
    res = {m: ber.simulate(h, code, 1.0, 2048, batch=1024, max_iter=50, msg_dtype=m, seed=4) for m in ("f32", "i8")}
    k32, k8 = res["f32"].frame_errors, res["i8"].frame_errors
    assert 20 < k32 < 2048 - 20
    lo8, hi8 = ber.wilson(k8, 2048)
    lo32, hi32 = ber.wilson(k32, 2048)
    assert lo8 <= hi32 and lo32 <= hi8, (k8, k32)
