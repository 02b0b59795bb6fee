"""FP16 and BF16 message storage vs the oracle with the same storage format.

The GPU computes each message in FP32 and rounds it to binary16 or bfloat16
(nearest, ties to even); the oracle computes it in FP64 and rounds it the same
way. A GPU value must be the correct rounding of some value within the FP32
path's message error of the oracle's unrounded message u: since rounding is
monotone, it lies between the roundings of u - tol and u + tol. Where the
format's spacing is wide against that error, this allows only the two
neighbours around a midpoint; at small magnitudes binary16's spacing (6e-8
below 6.1e-5) is finer than the product-form kernel's absolute error, and
more than one step may separate the two. The lock-step test checks this pass
by pass from the GPU's own previous messages.
"""

import numpy as np
import pytest

from paper_1609_01567_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# bound on the FP32 path's error in an unrounded message computed from the
# same previous messages: about five times the worst measured in the FP32
# lock-step test (5.8e-6)
MSG_TOL_ABS, MSG_TOL_REL = 3e-5, 1e-5


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
    cw = I.encode_ira(code, I.random_info(600, code.k, seed=1600))
    llr = I.gaussian_llr(cw, I.sigma2_from_ebn0(2.0, code.rate), seed=1601)
    return code, cw, llr


def gpu_decode(ldpc, handle, llr, max_iter, fmt, **kw):
    out = ldpc.ldpc_decode(handle, torch.from_numpy(np.ascontiguousarray(llr, dtype=np.float32)).cuda(), max_iter,
                           msg_dtype=fmt, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def ordered(x, fmt):
    """Integers in the order of the format's values (+0 and -0 both 0), so
    that neighbouring values differ by one."""
    x = np.asarray(x, dtype=np.float64)
    if fmt == "f16":
        b = x.astype(np.float16).view(np.uint16).astype(np.int64)
        mag, neg = b & 0x7FFF, (b >> 15) & 1
    else:
        b = (x.astype(np.float32).view(np.uint32) >> 16).astype(np.int64)
        mag, neg = b & 0x7FFF, (b >> 15) & 1
    return np.where(neg == 1, -mag, mag)


def on_grid(x, fmt):
    x = np.asarray(x, dtype=np.float64)
    if fmt == "f16":
        return np.array_equal(x.astype(np.float16).astype(np.float64), x)
    f = x.astype(np.float32)
    return np.array_equal(f.astype(np.float64), x) and not np.any(f.view(np.uint32) & 0xFFFF)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("rule,alpha,beta", [("sum_product", 1.0, 0.0), ("min_sum", 0.8, 0.2)])
def test_16_bit_lock_step_passes_n1008(ldpc, oracle_mod, n1008, fmt, rule, alpha, beta):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    kw = dict(rule=rule, rule_alpha=alpha, rule_beta=beta)
    okw = dict(rule="sp" if rule == "sum_product" else "min_sum", alpha=alpha, beta=beta, n_threads=8)
    v_of_edge = oracle_mod.address_iterators(code)["v"]
    lam = llr.astype(np.float64)
    prev_r = None
    n_off = n_multi = n_total = 0
    for t in range(0, 41, 4):
        if t > 0:
            prev_r = gpu_decode(ldpc, h, llr, t - 1, fmt, early_exit=False, want_r=True, **kw)["r"].astype(np.float64)
        got = gpu_decode(ldpc, h, llr, t, fmt, early_exit=False, want_r=True, **kw)
        ref = oracle_mod.sp_pass(code, lam, prev_r, msg=fmt, **okw)
        raw = oracle_mod.sp_pass(code, lam, prev_r, **okw)
        g, o, u = got["r"].astype(np.float64), ref["r"], raw["r"]
        assert on_grid(g, fmt) and on_grid(o, fmt), t
        off = g != o
        # a differing value is the rounding of a value within the FP32 error
        # of the unrounded message
        uu, gg = u[off], g[off]
        tol = MSG_TOL_ABS + MSG_TOL_REL * np.abs(uu)
        lo = np.array([oracle_mod.store(x, fmt) for x in uu - tol])
        hi = np.array([oracle_mod.store(x, fmt) for x in uu + tol])
        bad = (gg < lo) | (gg > hi)
        assert not bad.any(), (t, uu[bad][:5], gg[bad][:5], o[off][bad][:5])
        steps = np.abs(ordered(gg, fmt) - ordered(o[off], fmt))
        n_off += int(off.sum())
        n_multi += int((steps > 1).sum())
        n_total += off.size
        # posteriors: the sum of the stored messages, each differing value
        # moving its bit's posterior by the difference
        per_bit = np.zeros_like(got["post"], dtype=np.float64)
        for f in np.flatnonzero(off.any(axis=1)):
            np.add.at(per_bit[f], v_of_edge[off[f]], np.abs(g[f][off[f]] - o[f][off[f]]))
        dpost = np.abs(got["post"].astype(np.float64) - ref["post"])
        assert np.all(dpost <= 1e-4 * np.abs(ref["post"]) + 1e-4 + per_bit + 1e-6), (t, float(dpost.max()))
    assert n_off <= 1e-2 * n_total, (n_off, n_total)
    print(f"{fmt} lock-step {rule}: {n_off} of {n_total} stored values differ ({n_multi} by more than one step)")


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_16_bit_full_decode_n1008(ldpc, oracle_mod, n1008, fmt):
    """End to end: nearly every frame decodes to the bits and iteration count
    of the oracle with the same storage; a frame may part ways after a
    midpoint message."""
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    got = gpu_decode(ldpc, h, llr, 50, fmt)
    ref = oracle_mod.decode(code, llr.astype(np.float64), 50, n_threads=8, msg=fmt)
    same = (got["bits"] == ref["bits"]).all(axis=1) & (got["iters"] == ref["iters"]) & (got["ok"] == ref["ok"])
    assert same.mean() >= 0.97, np.flatnonzero(~same)[:10]
    assert (ref["ok"] == 1).mean() > 0.8


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_16_bit_fer_against_the_oracle_with_the_same_storage(ldpc, oracle_mod, fmt):
    from paper_1609_01567_gb300 import ber
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    frames, ebn0, seed = 3000, 1.5, 9
    lam = oracle_mod.gen_awgn(seed, 0, frames, code.n, I.sigma2_from_ebn0(ebn0, code.rate))
    ref = oracle_mod.decode(code, lam, 50, want_post=False, n_threads=16, msg=fmt)
    k_ref = int(ref["bits"].any(axis=1).sum())
    c = ber.simulate(h, code, ebn0, frames, batch=512, max_iter=50, msg_dtype=fmt, seed=seed)
    assert 30 < k_ref < frames - 30
    assert abs(c.frame_errors - k_ref) <= max(4, k_ref // 20), (c.frame_errors, k_ref)
