"""GPU (C ABI) vs the FP64 oracle, element by element, on the same seeded LLRs.

LLRs are drawn on the CPU (numpy PCG64 noise, `inputs.gaussian_llr`) and fed
to both sides, so no oracle input comes from the CUDA path. The on-device
generator is checked separately against the oracle's generator.
"""
import math

import numpy as np
import pytest

from paper_1609_01567_gb300 import inputs as I
from tests.parity import close, compare_decodes, near_zero_frames

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


def gpu_decode(ldpc, handle, llr, max_iter, **kw):
    out = ldpc.ldpc_decode(handle, torch.from_numpy(np.ascontiguousarray(llr, dtype=np.float32)).cuda(), max_iter, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def frames_of(code, n_frames, ebn0, seed):
    cw = I.encode_ira(code, I.random_info(n_frames, code.k, seed=seed))
    llr = I.gaussian_llr(cw, I.sigma2_from_ebn0(ebn0, code.rate), seed=seed + 1)
    return cw, llr


# --- generator ------------------------------------------------------------------

def test_philox_blocks_bit_exact(ldpc, oracle_mod):
    for key0, key1, ctr0, ctr1 in ((0, 0, 0, 0), (123456789, 42, 10 ** 15, 7), (2 ** 64 - 1, 2 ** 63, 2 ** 64 - 5, 1)):
        got = ldpc.ldpc_philox4x64_10(key0, key1, ctr0, ctr1, 1000).cpu().numpy().view(np.uint64)
        want = oracle_mod.philox_blocks(key0, key1, ctr0, ctr1, 1000)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("n,frames,offset", [(1008, 7, 0), (37, 33, 5), (64800, 3, 1000)])
def test_awgn_generator_matches_oracle(ldpc, oracle_mod, n, frames, offset):
    s2 = I.sigma2_from_ebn0(1.0, 0.5)
    rng = np.random.default_rng(n)
    cw = rng.integers(0, 2, size=(frames, n), dtype=np.uint8)
    got = ldpc.ldpc_gen_awgn(77, offset, frames, n, s2, torch.from_numpy(cw).cuda()).cpu().numpy()
    want = oracle_mod.gen_awgn(77, offset, frames, n, s2, cw)
    # float Box-Muller vs FP64: a few ulp of the noise sample, scaled by 2/sigma^2
    scale = 2.0 / s2 * (1.0 + math.sqrt(s2) * 6.0)
    np.testing.assert_allclose(got, want, rtol=2e-6, atol=2e-6 * scale)
    zero = ldpc.ldpc_gen_awgn(77, offset, frames, n, s2).cpu().numpy()
    np.testing.assert_allclose(zero, oracle_mod.gen_awgn(77, offset, frames, n, s2), rtol=2e-6, atol=2e-6 * scale)


# --- worked example and closed forms ------------------------------------------

def test_code_14_7_matches_oracle(ldpc, oracle_mod):
    code = I.code_14_7()
    h = ldpc.code_from_inputs(code)
    rng = np.random.default_rng(0)
    llr = rng.normal(-1.0, 1.6, size=(40, 14)).astype(np.float32)
    for max_iter, early in ((0, False), (3, False), (20, True)):
        got = gpu_decode(ldpc, h, llr, max_iter, early_exit=early)
        ref = oracle_mod.decode(code, llr.astype(np.float64), max_iter, early_exit=early)
        bad, exempt = compare_decodes(got, ref)
        assert bad.size == 0, (max_iter, bad)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7, 8, 9, 16, 31, 32, 33, 96, 200])
def test_single_parity_check_any_degree(ldpc, oracle_mod, d):
    """One check of degree d: every degree bin, closed-form pinned oracle."""
    code = I.coo_code(1, d, [0] * d, list(range(d)))
    h = ldpc.code_from_inputs(code)
    rng = np.random.default_rng(d)
    llr = rng.normal(0.0, 3.0, size=(70, d)).astype(np.float32)
    llr[0, 0] = 1e-7  # a dominant phi term beside small ones
    llr[0, 1:] = 30.0
    got = gpu_decode(ldpc, h, llr, 0, early_exit=False)
    ref = oracle_mod.decode(code, llr.astype(np.float64), 0, early_exit=False)
    assert close(got["post"], ref["post"]).all(), np.abs(got["post"] - ref["post"]).max()


@pytest.mark.parametrize("seed", range(4))
def test_tree_codes(ldpc, oracle_mod, seed):
    code = I.tree_code(18, seed=seed, max_check_degree=5)
    h = ldpc.code_from_inputs(code)
    llr = np.random.default_rng(seed).normal(0.0, 2.0, size=(50, code.n)).astype(np.float32)
    got = gpu_decode(ldpc, h, llr, code.n, early_exit=False)
    ref = oracle_mod.decode(code, llr.astype(np.float64), code.n, early_exit=False)
    bad, _ = compare_decodes(got, ref)
    assert bad.size == 0


def test_degenerate_nodes(ldpc, oracle_mod):
    """Degree-1 checks, an empty check, an isolated variable, zero LLRs."""
    code = I.coo_code(4, 5, [0, 1, 1, 3, 3], [0, 1, 2, 2, 3])
    h = ldpc.code_from_inputs(code)
    llr = np.array([[1.5, -0.5, 0.0, 2.0, 0.0], [0.0, 0.0, 0.0, 0.0, 0.0], [-3.0, 2.0, 0.25, -1.0, 4.0]],
                   dtype=np.float32)
    for early in (False, True):
        got = gpu_decode(ldpc, h, llr, 4, early_exit=early)
        ref = oracle_mod.decode(code, llr.astype(np.float64), 4, early_exit=early)
        assert close(got["post"], ref["post"]).all()
        np.testing.assert_array_equal(got["bits"], ref["bits"])
        np.testing.assert_array_equal(got["iters"], ref["iters"])
        np.testing.assert_array_equal(got["ok"], ref["ok"])


# --- the small workload: n = 1008, 1000 frames, 2 dB, max_iter 50, early stop ----

@pytest.fixture(scope="module")
def n1008():
    code = I.small_code_n1008()
    cw, llr = frames_of(code, 1000, 2.0, seed=1000)
    return code, cw, llr


def test_n1008_full_decode_matches_oracle(ldpc, oracle_mod, n1008):
    """The n = 1008 workload end to end: decisions, iteration counts and
    syndrome flags of every frame equal the oracle's (frames with a posterior
    within tolerance of 0 are logged instead), and posteriors match within
    the stated tolerance on frames that stop within 20 iterations. Longer
    trajectories accumulate FP32 rounding over many passes; they are checked
    pass by pass in test_lock_step_every_pass_n1008."""
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    got = gpu_decode(ldpc, h, llr, 50)
    ref = oracle_mod.decode(code, llr.astype(np.float64), 50, n_threads=8)
    same = (got["bits"] == ref["bits"]).all(axis=1) & (got["iters"] == ref["iters"]) & (got["ok"] == ref["ok"])
    exempt = near_zero_frames(ref["post"])
    diff = np.flatnonzero(~same & ~exempt)
    detail = [(int(f), int(got["iters"][f]), int(ref["iters"][f]), int(got["ok"][f]),
               int((got["bits"][f] != ref["bits"][f]).sum())) for f in diff[:10]]
    assert diff.size == 0, f"frames off the oracle (f, it_gpu, it_orc, ok_gpu, dbits): {detail}"
    short = ref["iters"] <= 20
    post_ok = close(got["post"], ref["post"]).all(axis=1)
    bad = np.flatnonzero(short & ~post_ok & ~exempt)
    assert bad.size == 0, [(int(f), float(np.abs(got["post"][f] - ref["post"][f]).max())) for f in bad[:10]]
    assert (ref["ok"] == 1).mean() > 0.8 and short.mean() > 0.8
    print(f"n1008: {len(same)} frames, {int(exempt.sum())} exempt (posterior near 0), "
          f"{int((~short).sum())} longer than 20 iterations")


@pytest.mark.parametrize("n_frames", [1, 31, 33, 64, 65, 129, 1000])
def test_n1008_ragged_batches(ldpc, oracle_mod, n1008, n_frames):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    sub = llr[:n_frames]
    got = gpu_decode(ldpc, h, sub, 8, early_exit=False)
    ref = oracle_mod.decode(code, sub.astype(np.float64), 8, early_exit=False, n_threads=8)
    bad, _ = compare_decodes(got, ref)
    assert bad.size == 0, bad[:10]


def test_lock_step_every_pass_n1008(ldpc, oracle_mod, n1008):
    """Every pass of every frame (51 passes, 1000 frames), each started from
    the GPU's own messages of the previous pass, equals the oracle's pass.

    Messages r get atol 1e-4: the GPU forms q = APP - r from its FP32
    posterior, whose rounding (up to ~1.5e-5 at |APP| ~ 200) reaches every
    output of a check through a rule that is 1-Lipschitz in each input."""
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    prev_r = None
    lam = llr.astype(np.float64)
    worst_post = worst_r = 0.0
    for t in range(51):
        got = gpu_decode(ldpc, h, llr, t, early_exit=False, want_r=True)
        ref = oracle_mod.sp_pass(code, lam, prev_r, n_threads=8)
        okp = close(got["post"], ref["post"])
        okr = close(got["r"], ref["r"], atol=1e-4)
        assert okp.all(), (t, np.argwhere(~okp)[:5].tolist(), float(np.abs(got["post"] - ref["post"]).max()))
        assert okr.all(), (t, float(np.abs(got["r"] - ref["r"]).max()))
        worst_post = max(worst_post, float(np.abs(got["post"] - ref["post"]).max()))
        worst_r = max(worst_r, float(np.abs(got["r"] - ref["r"]).max()))
        prev_r = got["r"].astype(np.float64)
    print(f"lock-step: worst |dpost| {worst_post:.2e}, worst |dr| {worst_r:.2e}")


def test_prefix_property_and_symmetry_on_gpu(ldpc, n1008):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    full = gpu_decode(ldpc, h, llr, 30)
    part = gpu_decode(ldpc, h, llr, 5)
    early = full["iters"] <= 5
    np.testing.assert_array_equal(part["iters"][early], full["iters"][early])
    np.testing.assert_array_equal(part["post"][early], full["post"][early])
    flip = gpu_decode(ldpc, h, llr * (1 - 2 * cw.astype(np.float32)), 30)
    np.testing.assert_array_equal(flip["iters"], full["iters"])
    np.testing.assert_array_equal(flip["bits"], full["bits"] ^ cw)
    np.testing.assert_array_equal(flip["post"], full["post"] * (1 - 2 * cw.astype(np.float32)))


@pytest.mark.parametrize("msg", ["f32", "f16", "bf16"])
def test_schedules_do_not_change_results(ldpc, n1008, msg):
    """Frames per lane, the check-kernel schedule, the two-stream split and the
    frame tiles are tuning knobs only: results are bit-identical."""
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    base = gpu_decode(ldpc, h, llr, 15, frames_per_lane=1, check_schedule=1, streams=1, msg_dtype=msg)
    for v, sched, nst, tile in ((2, 1, 1, 0), (4, 1, 1, 0), (2, 2, 1, 0), (4, 2, 1, 0), (4, 2, 2, 0), (8, 2, 2, 0),
                                (8, 1, 1, 0), (2, 2, 2, 0), (4, 2, 2, 256), (2, 2, 1, 64), (4, 2, 2, 128), (0, 0, 0, 0)):
        other = gpu_decode(ldpc, h, llr, 15, frames_per_lane=v, check_schedule=sched, streams=nst, tile_frames=tile,
                           msg_dtype=msg)
        for k in ("bits", "iters", "ok", "post"):
            np.testing.assert_array_equal(other[k], base[k],
                                          err_msg=f"V={v} schedule={sched} streams={nst} tile={tile} {k}")


def test_host_entry_point_matches_device_entry_point(ldpc, n1008):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    dev = gpu_decode(ldpc, h, llr[:300], 12)
    host = ldpc.ldpc_decode_host(h, llr[:300], 12, want_post=True)
    for k in ("bits", "iters", "ok", "post"):
        np.testing.assert_array_equal(host[k], dev[k])


# --- the large workload: n = 64800, 256 frames, 10 fixed iterations ------------------

@pytest.fixture(scope="module")
def n64800():
    code = I.large_code_n64800()
    cw, llr = frames_of(code, 256, 1.0, seed=64800)
    return code, cw, llr


def test_n64800_full_size_sampled_frames(ldpc, oracle_mod, n64800):
    """The benchmark's launch configuration (256 frames, max_iter 10 fixed):
    sampled frames against the oracle, all frames against the exact
    codeword sign symmetry."""
    code, cw, llr = n64800
    h = ldpc.code_from_inputs(code)
    got = gpu_decode(ldpc, h, llr, 10, early_exit=False)
    sample = np.array([0, 1, 77, 128, 200, 255])
    ref = oracle_mod.decode(code, llr[sample].astype(np.float64), 10, early_exit=False, n_threads=8)
    sub = {k: v[sample] for k, v in got.items()}
    bad, exempt = compare_decodes(sub, ref, frames=sample)
    assert bad.size == 0, (bad, exempt)
    flip = gpu_decode(ldpc, h, llr * (1 - 2 * cw.astype(np.float32)), 10, early_exit=False)
    np.testing.assert_array_equal(flip["bits"], got["bits"] ^ cw)
    np.testing.assert_array_equal(flip["ok"], got["ok"])


def test_fixed_decodes_without_posteriors_give_the_same_bits(ldpc, n1008, n64800):
    """Fixed-iteration decodes that skip the posteriors take their hard
    decisions from the last bit pass's decision words instead of the APP
    array; both give the same bits (the benchmark's configuration, ragged
    batches, every frames-per-lane width, one or two streams)."""
    for code, llr in ((n64800[0], n64800[2]), (n1008[0], n1008[2])):
        h = ldpc.code_from_inputs(code)
        for f, kw in ((256, {}), (256, dict(streams=1)), (37, {}), (300, dict(frames_per_lane=1)),
                      (200, dict(frames_per_lane=2, streams=2)), (1, {})):
            with_post = gpu_decode(ldpc, h, llr[:f], 7, early_exit=False, **kw)
            words = gpu_decode(ldpc, h, llr[:f], 7, early_exit=False, want_post=False, **kw)
            for k in ("bits", "iters", "ok"):
                np.testing.assert_array_equal(words[k], with_post[k], err_msg=f"{code.name} F={f} {kw} {k}")


def test_offsets_past_two_to_the_32(ldpc, oracle_mod):
    """Message offsets past 2^32: n = 262144 (E = 1,048,575) with 8192 frames
    in one chunk puts slot * Fp up to 8.6e9 (about 71 GB on the device). Three
    passes; sampled frames, the last one included (highest offsets), against
    the oracle."""
    from paper_1609_01567_gb300 import sweep
    code = sweep.stand_in_code(262144)
    h = ldpc.code_from_inputs(code)
    F = 8192
    assert code.n_edges * F > 2 ** 32
    llr = ldpc.ldpc_gen_awgn(5, 0, F, code.n, I.sigma2_from_ebn0(1.5, code.rate))
    out = ldpc.ldpc_decode(h, llr, 2, early_exit=False)
    torch.cuda.synchronize()
    sample = torch.tensor([0, 1, 4095, 8190, 8191])
    got = {k: v[sample.to(v.device)].cpu().numpy() for k, v in out.items()}
    lam = llr[sample.to(llr.device)].cpu().numpy().astype(np.float64)
    del out, llr
    torch.cuda.empty_cache()
    ref = oracle_mod.decode(code, lam, 2, early_exit=False, n_threads=8)
    bad, exempt = compare_decodes(got, ref, frames=sample.numpy())
    assert bad.size == 0, (bad, exempt)


@pytest.fixture(scope="module")
def n64800_r56():
    code = I.mixed_code(7)  # n = 64800, rate 5/6, 10,800 checks of degree 17-18
    llr = I.gaussian_llr(np.zeros((256, code.n), np.uint8), I.sigma2_from_ebn0(2.9, code.rate), seed=5656)
    return code, llr


@pytest.mark.parametrize("rule", ["sum_product", "min_sum"])
def test_high_rate_checks_lock_step(ldpc, oracle_mod, n64800_r56, rule):
    """Checks of degree 17-18 in a code with many of them run in the
    pipelined kernel with 18 slots: three passes at 256 frames, sampled frames against the
    oracle from the GPU's own messages (sum-product and offset/normalised
    min-sum)."""
    code, llr = n64800_r56
    h = ldpc.code_from_inputs(code)
    info = ldpc.ldpc_code_info(h)
    assert info["check_bin_count"][4] == code.m and code.m >= 2048
    kw = dict(rule=rule, rule_alpha=0.85, rule_beta=0.1) if rule == "min_sum" else {}
    okw = dict(rule="min_sum", alpha=0.85, beta=0.1) if rule == "min_sum" else {}
    sample = np.array([0, 5, 128, 255])
    prev_r = None
    for t in range(3):
        got = gpu_decode(ldpc, h, llr, t, early_exit=False, want_r=True, **kw)
        ref = oracle_mod.sp_pass(code, llr[sample].astype(np.float64), prev_r, n_threads=8, **okw)
        assert close(got["post"][sample], ref["post"]).all(), (t, np.abs(got["post"][sample] - ref["post"]).max())
        assert close(got["r"][sample], ref["r"], atol=1e-4).all(), (t, np.abs(got["r"][sample] - ref["r"]).max())
        prev_r = got["r"][sample].astype(np.float64)


def test_high_rate_results_do_not_depend_on_layout_or_batch(ldpc, n64800_r56):
    """The degree-18 checks' results are the same at four, two and one
    frames per lane, on one or two streams, and for a frame decoded alone or
    in a batch of 256. Batches of 64-frame groups run the pipelined kernel
    with 18 slots; a batch of 20 frames (one 32-frame group) runs the staged
    product-form kernel at one frame per lane, the same operations in the
    same order, so its frames equal the batch's bit for bit."""
    code, llr = n64800_r56
    h = ldpc.code_from_inputs(code)
    base = gpu_decode(ldpc, h, llr, 8, early_exit=False)
    for kw in (dict(frames_per_lane=2), dict(frames_per_lane=1, streams=1), dict(streams=1)):
        other = gpu_decode(ldpc, h, llr, 8, early_exit=False, **kw)
        for k in ("bits", "iters", "ok", "post"):
            np.testing.assert_array_equal(other[k], base[k], err_msg=f"{kw} {k}")
    for nf in (37, 20):
        part = gpu_decode(ldpc, h, llr[:nf], 8, early_exit=False)
        for k in ("bits", "iters", "ok", "post"):
            np.testing.assert_array_equal(part[k], base[k][:nf], err_msg=f"{nf} frames {k}")


@pytest.mark.parametrize("rule", ["sum_product", "min_sum"])
def test_wide_check_lock_step_and_layouts(ldpc, oracle_mod, rule):
    """A code with one check of degree 96 (and a variable of degree 64): the
    wide check runs a CTA per frame group, its warps splitting the inputs.
    Four passes at 256 frames on sampled frames against the oracle, and the
    same results at every frames-per-lane width and on one or two streams."""
    code = I.mixed_code(4)
    h = ldpc.code_from_inputs(code)
    assert ldpc.ldpc_code_info(h)["check_bin_count"][5] == 1
    llr = I.gaussian_llr(np.zeros((256, code.n), np.uint8), I.sigma2_from_ebn0(2.4, code.rate), seed=9696)
    kw = dict(rule=rule, rule_alpha=0.8, rule_beta=0.1) if rule == "min_sum" else {}
    okw = dict(rule="min_sum", alpha=0.8, beta=0.1) if rule == "min_sum" else {}
    sample = np.array([0, 63, 64, 200, 255])
    prev_r = None
    for t in range(4):
        got = gpu_decode(ldpc, h, llr, t, early_exit=False, want_r=True, **kw)
        ref = oracle_mod.sp_pass(code, llr[sample].astype(np.float64), prev_r, n_threads=8, **okw)
        assert close(got["post"][sample], ref["post"]).all(), (t, np.abs(got["post"][sample] - ref["post"]).max())
        assert close(got["r"][sample], ref["r"], atol=1e-4).all(), (t, np.abs(got["r"][sample] - ref["r"]).max())
        prev_r = got["r"][sample].astype(np.float64)
    base = gpu_decode(ldpc, h, llr, 12, **kw)
    for lay in (dict(frames_per_lane=2), dict(frames_per_lane=1), dict(streams=1), dict(frames_per_lane=8)):
        other = gpu_decode(ldpc, h, llr, 12, **kw, **lay)
        for k in ("bits", "iters", "ok", "post"):
            np.testing.assert_array_equal(other[k], base[k], err_msg=f"{lay} {k}")


@pytest.mark.parametrize("rule", ["sum_product", "min_sum"])
def test_short_high_rate_code_ring_and_register_kernels(ldpc, oracle_mod, rule):
    """A short rate-5/6 code (95 checks of degree 17-18): batches of 64-frame
    groups run the 18-slot ring kernel, a 20-frame batch and check_schedule 1
    the register kernel (32 slots, one frame per lane, direct loads). Same
    results bit for bit, and the oracle's on every frame that stops within
    12 iterations (min-sum: the offset/normalised rule)."""
    code = I.mixed_code(0)  # n = 576, rate 5/6
    h = ldpc.code_from_inputs(code)
    assert ldpc.ldpc_code_info(h)["check_bin_count"][4] == code.m
    kw = dict(rule=rule, rule_alpha=0.85, rule_beta=0.1) if rule == "min_sum" else {}
    okw = dict(rule="min_sum", alpha=0.85, beta=0.1) if rule == "min_sum" else {}
    llr = I.gaussian_llr(np.zeros((256, code.n), np.uint8), I.sigma2_from_ebn0(4.0, code.rate), seed=576)
    base = gpu_decode(ldpc, h, llr, 20, **kw)
    reg = gpu_decode(ldpc, h, llr, 20, check_schedule=1, **kw)
    part = gpu_decode(ldpc, h, llr[:20], 20, **kw)
    for k in ("bits", "iters", "ok", "post"):
        np.testing.assert_array_equal(reg[k], base[k], err_msg=f"register kernel {k}")
        np.testing.assert_array_equal(part[k], base[k][:20], err_msg=f"20 frames {k}")
    ref = oracle_mod.decode(code, llr.astype(np.float64), 20, n_threads=8, **okw)
    bad, exempt = compare_decodes(base, ref)
    short = ref["iters"] <= 12
    assert short.mean() > 0.5 and not np.isin(bad, np.flatnonzero(short)).any(), bad


def test_checks_of_degree_9_to_12_in_twelve_slots(ldpc, oracle_mod):
    """A bin of checks of degree 9-16 whose largest degree is 12 runs in 12
    slots instead of 16; padding slots are exact no-ops, so the results equal
    the 16-slot kernel's (check_schedule 1) bit for bit, and the oracle's."""
    code = I.mixed_code(1)  # n = 1152, rate 3/4, checks of degree 11-12
    h = ldpc.code_from_inputs(code)
    assert ldpc.ldpc_code_info(h)["check_bin_count"][3] == code.m
    llr = I.gaussian_llr(np.zeros((256, code.n), np.uint8), I.sigma2_from_ebn0(3.3, code.rate), seed=1212)
    base = gpu_decode(ldpc, h, llr, 20)
    slots16 = gpu_decode(ldpc, h, llr, 20, check_schedule=1)
    for k in ("bits", "iters", "ok", "post"):
        np.testing.assert_array_equal(slots16[k], base[k], err_msg=k)
    ref = oracle_mod.decode(code, llr.astype(np.float64), 20, n_threads=8)
    bad, exempt = compare_decodes(base, ref)
    short = ref["iters"] <= 12
    assert not np.isin(bad, np.flatnonzero(short)).any(), bad


@pytest.mark.parametrize("msg", ["f16", "bf16", "i8"])
def test_new_check_paths_in_every_message_format(ldpc, msg):
    """The 12-slot, 18-slot (high-rate) and wide-check paths with 16-bit
    and int8 messages: the same results as the direct-load kernels (the
    staged product form for the high-rate checks) at one frame per lane on
    one stream, and the same codeword as the FP32 decode on nearly every
    frame that FP32 corrects."""
    for idx, ebn0 in ((1, 3.6), (4, 2.8), (7, 3.1)):  # n = 1152 r 3/4, n = 8192 with a degree-96 check, n = 64800 r 5/6
        code = I.mixed_code(idx)
        h = ldpc.code_from_inputs(code)
        llr = I.gaussian_llr(np.zeros((256, code.n), np.uint8), I.sigma2_from_ebn0(ebn0, code.rate), seed=77 + idx)
        base = gpu_decode(ldpc, h, llr, 15, msg_dtype=msg)
        other = gpu_decode(ldpc, h, llr, 15, msg_dtype=msg, frames_per_lane=1, check_schedule=1, streams=1)
        for k in ("bits", "iters", "ok", "post"):
            np.testing.assert_array_equal(other[k], base[k], err_msg=f"{code.name} {msg} {k}")
        f32 = gpu_decode(ldpc, h, llr, 15)
        conv = f32["ok"] == 1  # frames the FP32 decode corrects; the others part ways chaotically
        agree = ((base["bits"] == f32["bits"]).all(axis=1) & (base["ok"] == 1))[conv].mean()
        assert conv.mean() > 0.3 and agree >= 0.9, (code.name, msg, conv.mean(), agree)


def test_n64800_lock_step_two_passes(ldpc, oracle_mod, n64800):
    code, cw, llr = n64800
    h = ldpc.code_from_inputs(code)
    sub = llr[:8]
    prev_r = None
    for t in range(3):
        got = gpu_decode(ldpc, h, sub, t, early_exit=False, want_r=True)
        ref = oracle_mod.sp_pass(code, sub.astype(np.float64), prev_r, n_threads=8)
        assert close(got["post"], ref["post"]).all(), (t, np.abs(got["post"] - ref["post"]).max())
        prev_r = got["r"].astype(np.float64)


def test_profile_counts_launches(ldpc, n1008):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    ldpc.ldpc_prof_read(h, reset=True)
    gpu_decode(ldpc, h, llr[:128], 4, early_exit=False, profile=True)
    prof = ldpc.ldpc_prof_read(h, reset=True)
    assert prof["bit"]["launches"] == 5
    assert prof["check"]["launches"] >= 5
    assert prof["check"]["total_ms"] > 0.0


# --- min-sum family --------------------------------------------------------------

@pytest.mark.parametrize("d", [1, 2, 3, 5, 6, 7, 8, 16, 32, 33, 96])
def test_min_sum_single_check_any_degree(ldpc, oracle_mod, d):
    code = I.coo_code(1, d, [0] * d, list(range(d)))
    h = ldpc.code_from_inputs(code)
    llr = np.random.default_rng(d).normal(0.0, 3.0, size=(70, d)).astype(np.float32)
    llr[1, :] = llr[1, 0]  # ties between the two smallest magnitudes
    for alpha, beta in ((1.0, 0.0), (0.75, 0.0), (1.0, 0.5)):
        got = gpu_decode(ldpc, h, llr, 0, early_exit=False, rule="min_sum", rule_alpha=alpha, rule_beta=beta)
        ref = oracle_mod.decode(code, llr.astype(np.float64), 0, early_exit=False, rule="min_sum", alpha=alpha,
                                beta=beta)
        assert close(got["post"], ref["post"]).all(), (alpha, beta, np.abs(got["post"] - ref["post"]).max())


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (0.8, 0.0), (1.0, 0.3)])
def test_min_sum_n1008_matches_oracle(ldpc, oracle_mod, n1008, alpha, beta):
    """End to end on frames that stop within 20 iterations; longer
    trajectories are checked pass by pass in the lock-step test below."""
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    got = gpu_decode(ldpc, h, llr, 50, rule="min_sum", rule_alpha=alpha, rule_beta=beta)
    ref = oracle_mod.decode(code, llr.astype(np.float64), 50, n_threads=8, rule="min_sum", alpha=alpha, beta=beta)
    same = (got["bits"] == ref["bits"]).all(axis=1) & (got["iters"] == ref["iters"]) & (got["ok"] == ref["ok"])
    exempt = near_zero_frames(ref["post"])
    short = ref["iters"] <= 20
    assert np.all(same | exempt | ~short), np.flatnonzero(~same & ~exempt & short)[:10]
    assert close(got["post"], ref["post"]).all(axis=1)[short & ~exempt].all()
    assert short.mean() > 0.5 and same.mean() > 0.98


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (0.8, 0.2)])
def test_min_sum_lock_step_every_pass_n1008(ldpc, oracle_mod, n1008, alpha, beta):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    kw = dict(rule="min_sum", rule_alpha=alpha, rule_beta=beta)
    prev_r = None
    lam = llr.astype(np.float64)
    for t in range(0, 51, 5):
        if t > 0:
            prev = gpu_decode(ldpc, h, llr, t - 1, early_exit=False, want_r=True, **kw)
            prev_r = prev["r"].astype(np.float64)
        got = gpu_decode(ldpc, h, llr, t, early_exit=False, want_r=True, **kw)
        ref = oracle_mod.sp_pass(code, lam, prev_r, n_threads=8, rule="min_sum", alpha=alpha, beta=beta)
        assert close(got["post"], ref["post"]).all(), (t, float(np.abs(got["post"] - ref["post"]).max()))
        assert close(got["r"], ref["r"], atol=1e-4).all(), (t, float(np.abs(got["r"] - ref["r"]).max()))


def test_min_sum_schedules_do_not_change_results(ldpc, n1008):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    kw = dict(rule="min_sum", rule_alpha=0.8)
    base = gpu_decode(ldpc, h, llr, 15, frames_per_lane=1, check_schedule=1, streams=1, **kw)
    for v, sched, nst in ((4, 2, 2), (2, 2, 1), (8, 1, 1)):
        other = gpu_decode(ldpc, h, llr, 15, frames_per_lane=v, check_schedule=sched, streams=nst, **kw)
        for k in ("bits", "iters", "ok", "post"):
            np.testing.assert_array_equal(other[k], base[k], err_msg=f"V={v} schedule={sched} streams={nst} {k}")


# --- degree-adaptive min-sum (rule "min_sum_adaptive") ---------------------------

def degree_tables(n):
    """A scale and an offset for every degree below n, each differing from its
    neighbours', so that a table read at the wrong degree shows."""
    d = np.arange(n)
    return 0.55 + 0.04 * ((d * 37) % 11), 0.1 * (d % 4) + 0.02 * (d % 3)


def test_adaptive_min_sum_checks_of_every_bin(ldpc, oracle_mod):
    """Disjoint checks of degrees spanning every degree bin (and past the
    table's end) after the first check pass, for each frames-per-lane width."""
    degs = [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 16, 17, 31, 32, 33, 64, 96]
    rows = np.repeat(np.arange(len(degs)), degs)
    cols = np.arange(rows.size)
    code = I.coo_code(len(degs), int(rows.size), rows.tolist(), cols.tolist())
    h = ldpc.code_from_inputs(code)
    alpha, beta = degree_tables(40)
    ldpc.ldpc_code_set_rule_table(h, alpha, beta)
    llr = np.random.default_rng(11).normal(0.0, 3.0, size=(300, code.n)).astype(np.float32)
    ref = oracle_mod.decode(code, llr.astype(np.float64), 0, early_exit=False, rule="min_sum_adaptive",
                            alpha_by_degree=alpha.astype(np.float32), beta_by_degree=beta.astype(np.float32))
    for v in (1, 2, 4):
        got = gpu_decode(ldpc, h, llr, 0, early_exit=False, rule="min_sum_adaptive", frames_per_lane=v)
        assert close(got["post"], ref["post"]).all(), (v, np.abs(got["post"] - ref["post"]).max())


def test_adaptive_min_sum_lock_step_n1008(ldpc, oracle_mod, n1008):
    """Check degrees 5 and 6 with their own scale and offset, pass by pass
    from the GPU's own messages, and end to end on frames that stop early."""
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    alpha, beta = [1.0] * 5 + [0.8, 0.9], [0.0] * 5 + [0.05, 0.15]
    ldpc.ldpc_code_set_rule_table(h, alpha, beta)
    kw = dict(rule="min_sum_adaptive")
    okw = dict(rule="min_sum_adaptive", alpha_by_degree=np.float32(alpha), beta_by_degree=np.float32(beta))
    lam = llr.astype(np.float64)
    prev_r = None
    for t in range(0, 31, 5):
        if t > 0:
            prev_r = gpu_decode(ldpc, h, llr, t - 1, early_exit=False, want_r=True, **kw)["r"].astype(np.float64)
        got = gpu_decode(ldpc, h, llr, t, early_exit=False, want_r=True, **kw)
        ref = oracle_mod.sp_pass(code, lam, prev_r, n_threads=8, **okw)
        assert close(got["post"], ref["post"]).all(), (t, float(np.abs(got["post"] - ref["post"]).max()))
        assert close(got["r"], ref["r"], atol=1e-4).all(), (t, float(np.abs(got["r"] - ref["r"]).max()))
    got = gpu_decode(ldpc, h, llr, 50, **kw)
    ref = oracle_mod.decode(code, lam, 50, n_threads=8, **okw)
    same = (got["bits"] == ref["bits"]).all(axis=1) & (got["iters"] == ref["iters"]) & (got["ok"] == ref["ok"])
    short = ref["iters"] <= 20
    exempt = near_zero_frames(ref["post"])
    assert np.all(same | exempt | ~short), np.flatnonzero(~same & ~exempt & short)[:10]
    assert short.sum() >= 200, short.sum()  # enough frames compared end to end
    # a constant table is the plain normalised/offset rule, bit for bit
    ldpc.ldpc_code_set_rule_table(h, [0.8], [0.2])
    a = gpu_decode(ldpc, h, llr, 12, early_exit=False, **kw)
    b = gpu_decode(ldpc, h, llr, 12, early_exit=False, rule="min_sum", rule_alpha=0.8, rule_beta=0.2)
    for k in ("bits", "iters", "ok", "post"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_adaptive_min_sum_n64800_sampled_frames(ldpc, oracle_mod, n64800):
    """The large workload's launch shape (256 frames), two passes, sampled
    frames against the oracle from the GPU's own messages."""
    code, cw, llr = n64800
    h = ldpc.code_from_inputs(code)
    alpha, beta = [1.0] * 5 + [0.9, 0.75], [0.0] * 5 + [0.3, 0.05]
    ldpc.ldpc_code_set_rule_table(h, alpha, beta)
    okw = dict(rule="min_sum_adaptive", alpha_by_degree=np.float32(alpha), beta_by_degree=np.float32(beta))
    sample = np.array([0, 77, 200, 255])
    prev_r = None
    for t in range(2):
        got = gpu_decode(ldpc, h, llr, t, early_exit=False, want_r=True, rule="min_sum_adaptive")
        ref = oracle_mod.sp_pass(code, llr[sample].astype(np.float64), prev_r, n_threads=8, **okw)
        assert close(got["post"][sample], ref["post"]).all(), (t, np.abs(got["post"][sample] - ref["post"]).max())
        prev_r = got["r"][sample].astype(np.float64)


def test_adaptive_min_sum_needs_a_table(ldpc, n1008):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    with pytest.raises(ldpc.LdpcError) as e:
        gpu_decode(ldpc, h, llr[:32], 5, rule="min_sum_adaptive")
    assert "ldpc_code_set_rule_table" in str(e.value)


# --- sum-product with tabulated phi (rule "sp_table") ------------------------------

@pytest.mark.parametrize("d", [1, 2, 3, 6, 8, 17, 33, 96])
def test_table_rule_single_check_any_degree(ldpc, oracle_mod, d):
    code = I.coo_code(1, d, [0] * d, list(range(d)))
    h = ldpc.code_from_inputs(code)
    llr = np.random.default_rng(d + 100).normal(0.0, 3.0, size=(70, d)).astype(np.float32)
    llr[0, 0] = 1e-7
    llr[0, 1:] = 30.0
    got = gpu_decode(ldpc, h, llr, 0, early_exit=False, rule="sp_table")
    ref = oracle_mod.decode(code, llr.astype(np.float64), 0, early_exit=False, rule="sp_table")
    assert close(got["post"], ref["post"]).all(), np.abs(got["post"] - ref["post"]).max()


def test_table_rule_lock_step_n1008(ldpc, oracle_mod, n1008):
    """Every fifth pass of 51, from the GPU's own previous messages: the
    tabulated rule on the GPU (float chords, bucket chosen on the float
    value) equals the oracle's (chords in double)."""
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    lam = llr.astype(np.float64)
    prev_r = None
    for t in range(0, 51, 5):
        if t > 0:
            prev_r = gpu_decode(ldpc, h, llr, t - 1, early_exit=False, want_r=True, rule="sp_table")["r"]
            prev_r = prev_r.astype(np.float64)
        got = gpu_decode(ldpc, h, llr, t, early_exit=False, want_r=True, rule="sp_table")
        ref = oracle_mod.sp_pass(code, lam, prev_r, n_threads=8, rule="sp_table")
        assert close(got["post"], ref["post"]).all(), (t, float(np.abs(got["post"] - ref["post"]).max()))
        assert close(got["r"], ref["r"], atol=1e-4).all(), (t, float(np.abs(got["r"] - ref["r"]).max()))


def test_table_rule_schedules_and_limits(ldpc, n1008):
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    base = gpu_decode(ldpc, h, llr, 15, frames_per_lane=1, check_schedule=1, streams=1, rule="sp_table")
    for v, sched, nst in ((4, 2, 2), (2, 0, 1), (8, 0, 0)):
        other = gpu_decode(ldpc, h, llr, 15, frames_per_lane=v, check_schedule=sched, streams=nst, rule="sp_table")
        for k in ("bits", "iters", "ok", "post"):
            np.testing.assert_array_equal(other[k], base[k], err_msg=f"V={v} schedule={sched} streams={nst} {k}")
    assert (base["ok"] == 1).mean() > 0.7  # 15 iterations at 2 dB
    with pytest.raises(ldpc.LdpcError):
        gpu_decode(ldpc, h, llr[:4], 5, rule="sp_table", l_max=30.0)


def test_unaligned_caller_buffers(ldpc, n1008):
    """LLRs, decisions and posteriors at odd offsets take the scalar paths of
    the layout kernels and give the same results as aligned buffers."""
    code, cw, llr = n1008
    h = ldpc.code_from_inputs(code)
    sub = np.ascontiguousarray(llr[:70], dtype=np.float32)
    f, n = sub.shape
    base = gpu_decode(ldpc, h, sub, 12)
    lbuf = torch.zeros(f * n + 1, dtype=torch.float32, device="cuda")
    lbuf[1:] = torch.from_numpy(sub.reshape(-1)).cuda()
    out = {"bits": torch.zeros(f * n + 1, dtype=torch.uint8, device="cuda")[1:].view(f, n),
           "iters": torch.zeros(f, dtype=torch.int32, device="cuda"),
           "ok": torch.zeros(f, dtype=torch.uint8, device="cuda"),
           "post": torch.zeros(f * n + 1, dtype=torch.float32, device="cuda")[1:].view(f, n)}
    got = ldpc.ldpc_decode(h, lbuf[1:].view(f, n), 12, out=out)
    torch.cuda.synchronize()
    for k in ("bits", "iters", "ok", "post"):
        np.testing.assert_array_equal(got[k].cpu().numpy(), base[k], err_msg=k)


def test_batches_larger_than_one_chunk(ldpc, oracle_mod):
    """More frames than one device chunk (8192): the decode runs in chunks
    that reuse the workspace; every frame still equals the oracle."""
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    F = 8192 + 300
    llr = I.gaussian_llr(np.zeros((F, code.n), np.uint8), I.sigma2_from_ebn0(2.5, code.rate), seed=77)
    got = gpu_decode(ldpc, h, llr, 4)
    ref = oracle_mod.decode(code, llr.astype(np.float64), 4, n_threads=8)
    bad, _ = compare_decodes(got, ref)
    assert bad.size == 0, bad[:10]
