"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows. None of them compares the oracle with
itself: the expected values come from the paper's tables, from closed forms,
from brute force over all codewords, from numpy's independent Philox, or from
exact invariants of the sum-product rules.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_1609_01567_gb300 import inputs as I
from tests.paper_tables import table


# --- Tables 1-2 (Section III-B) --------------------------------------------------

def test_address_iterators_match_tables_1_and_2(oracle_mod):
    it = oracle_mod.address_iterators(I.code_14_7())
    for number in (1, 2):
        for name, want in table(number).items():
            np.testing.assert_array_equal(it[name], want, err_msg=f"Table {number} array {name}")


def test_example_code_edges_are_table_1():
    """The input module's copy of the (14,7) code is Table 1's v and c rows."""
    code = I.code_14_7()
    t1 = table(1)
    np.testing.assert_array_equal(code.cols, t1["v"])
    np.testing.assert_array_equal(code.rows, t1["c"])


# --- sigma^2 of the BER simulator (Section IV) -----------------------------------

@pytest.mark.parametrize("ebn0_db,rate,want", [
    (0.0, 0.5, 1.0),                                 # 1 / (2 * 1/2 * 1)
    (10.0, 0.5, 0.1),                                # 1 / (2 * 1/2 * 10)
    (0.0, 0.25, 2.0),                                # 1 / (2 * 1/4 * 1)
    (10.0, 1.0 / 3.0, 0.15),                         # 1 / (2 * 1/3 * 10)
    (3.0, 5.0 / 6.0, 0.3007123401763634),            # 1 / (5/3 * 1.99526231497) = 1 / 3.32543719161
    (20.0, 0.5, 0.01),
])
def test_sigma2_from_ebn0_hand_values(ebn0_db, rate, want):
    """Unit-energy BPSK: Es = 1, Eb = 1/R, sigma^2 = N0/2 = 1 / (2 R Eb/N0).
    The expected values are worked out by hand, so a wrong factor of 2, R or
    a dB conversion by 20 instead of 10 fails here (both sides of every
    parity test read this one function)."""
    assert I.sigma2_from_ebn0(ebn0_db, rate) == pytest.approx(want, rel=1e-12)


def test_code_14_7_rank_and_text_example(oracle_mod):
    """Section II-C: v0 joins c0, c2, c3, c5 and c3 joins v0, v4, v11, v12; k = 7."""
    code = I.code_14_7()
    h = code.dense()
    assert set(np.flatnonzero(h[:, 0])) == {0, 2, 3, 5}
    assert set(np.flatnonzero(h[3])) == {0, 4, 11, 12}
    words = oracle_mod.codewords_of(code)
    assert words.shape == (2 ** 7, 14)
    assert np.all(oracle_mod.syndrome_weight(code, words) == 0)
    assert len({w.tobytes() for w in words}) == 128


# --- syndrome and encoder (Section II-B: v is a codeword iff v H^T = 0) ----------

def test_syndrome_of_unit_vectors_is_column_weight(oracle_mod):
    code = I.small_code_n1008()
    eye = np.eye(code.n, dtype=np.uint8)[:50]
    colw = np.bincount(code.cols, minlength=code.n)[:50]
    np.testing.assert_array_equal(oracle_mod.syndrome_weight(code, eye), colw)


@pytest.mark.parametrize("which", ["n1008", "n64800"])
def test_encoded_words_have_zero_syndrome(oracle_mod, which):
    code = I.small_code_n1008() if which == "n1008" else I.large_code_n64800()
    cw = I.encode_ira(code, I.random_info(6, code.k, seed=11))
    assert np.all(oracle_mod.syndrome_weight(code, cw) == 0)
    bad = cw.copy()
    bad[:, 3] ^= 1
    assert np.all(oracle_mod.syndrome_weight(code, bad) == np.bincount(code.cols, minlength=code.n)[3])


def test_code_profiles():
    """Workload sizes: E = 2873 at n = 1008 and E = 194399 at n = 64800."""
    c1, c2 = I.small_code_n1008(), I.large_code_n64800()
    assert c1.n_edges == 2873 and c2.n_edges == 194399
    for c in (c1, c2):
        key = c.rows.astype(np.int64) * c.n + c.cols
        assert np.unique(key).size == key.size
    vd = np.bincount(c2.cols, minlength=c2.n)
    assert (vd == 8).sum() == 6480 and (vd == 3).sum() == 25920
    cd = np.bincount(c2.rows, minlength=c2.m)
    assert (cd == 6).sum() == 32399 and cd[0] == 5


# --- check rule: closed forms --------------------------------------------------

def test_single_parity_check_closed_form(oracle_mod):
    """Algorithm 1 (second half) on one check equals the exact parity posterior
    lambda_j - 2 atanh(prod_{j' != j} (-tanh(lambda_j'/2))), and brute force."""
    rng = np.random.default_rng(3)
    for d in (2, 3, 5, 8):
        code = I.coo_code(1, d, [0] * d, list(range(d)))
        lam = rng.normal(0.0, 2.5, size=(20, d))
        out = oracle_mod.decode(code, lam, 0, early_exit=False, l_max=60.0)
        t = -np.tanh(lam / 2.0)
        want = np.empty_like(lam)
        for j in range(d):
            prod = np.prod(np.delete(t, j, axis=1), axis=1)
            want[:, j] = lam[:, j] - 2.0 * np.arctanh(prod)
        np.testing.assert_allclose(out["post"], want, rtol=1e-11, atol=1e-11)
        words = oracle_mod.codewords_of(code)
        np.testing.assert_allclose(out["post"], oracle_mod.map_llr(words, lam), rtol=1e-9, atol=1e-9)


def test_degree_two_check_passes_clamped_message(oracle_mod):
    """phi is an involution, so a degree-2 check forwards sign(q) * clamp(|q|,
    phi(L_MAX), L_MAX): the saturation reading of the check rule."""
    code = I.coo_code(1, 2, [0, 0], [0, 1])
    lam = np.array([[0.5, 35.0], [0.5, -7.25], [-1.0, 3.0], [2.0, -50.0]])
    out = oracle_mod.decode(code, lam, 0, early_exit=False, l_max=20.0)
    want0 = lam[:, 0] + np.sign(lam[:, 1]) * np.minimum(np.abs(lam[:, 1]), 20.0)
    np.testing.assert_allclose(out["post"][:, 0], want0, rtol=1e-12)


def test_degree_one_check_and_isolated_nodes(oracle_mod):
    """Degree-1 check: empty product, r0 = 1, so r = -L_MAX. Degree-0 variable:
    APP = lambda; its tie APP = 0 decides 0 (Algorithm 5). Empty check: z = 0."""
    code = I.coo_code(3, 3, [0, 1], [0, 1])  # check 2 empty, variable 2 isolated
    lam = np.array([[1.5, -0.5, 0.0], [-3.0, 2.0, 0.25]])
    out = oracle_mod.decode(code, lam, 0, early_exit=False, l_max=20.0)
    np.testing.assert_allclose(out["post"], lam + np.array([-20.0, -20.0, 0.0]))
    assert out["bits"][0, 2] == 0 and out["bits"][1, 2] == 1
    assert np.all(out["ok"] == 1)


# --- whole decoder on cycle-free graphs: BP is exact ---------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_tree_decoder_equals_bitwise_map(oracle_mod, seed):
    code = I.tree_code(14 + seed, seed=seed)
    words = oracle_mod.codewords_of(code)
    rng = np.random.default_rng(100 + seed)
    lam = rng.normal(0.0, 2.0, size=(12, code.n))
    out = oracle_mod.decode(code, lam, code.n, early_exit=False, l_max=60.0)
    np.testing.assert_allclose(out["post"], oracle_mod.map_llr(words, lam), rtol=1e-9, atol=1e-9)


def test_repetition_code_sums_llrs(oracle_mod):
    """Checks v0 + vi = 0: every bit equals v0, so APP_j = sum of all LLRs."""
    n = 7
    code = I.coo_code(n - 1, n, [i - 1 for i in range(1, n)] * 2, [0] * (n - 1) + list(range(1, n)))
    lam = np.random.default_rng(5).normal(0.3, 1.5, size=(9, n))
    out = oracle_mod.decode(code, lam, 3, early_exit=False, l_max=60.0)
    np.testing.assert_allclose(out["post"], np.repeat(lam.sum(axis=1, keepdims=True), n, axis=1), rtol=1e-10)


# --- LLR rewrite vs the literal probability-domain algorithms ----------------------

@pytest.mark.parametrize("which", ["14_7", "ira40"])
def test_llr_oracle_matches_probability_domain(oracle_mod, which):
    code = I.code_14_7() if which == "14_7" else I.ira_code(40, 20, {3: 0.6, 4: 0.4}, seed=4)
    rng = np.random.default_rng(9)
    sigma2 = 0.9
    y = -1.0 + math.sqrt(sigma2) * rng.standard_normal((5, code.n))
    lit = oracle_mod.decode_probability_domain(code, y, sigma2, 4)
    lam = 2.0 * y / sigma2
    r_prev = None
    for p in range(5):
        st = oracle_mod.sp_pass(code, lam, r_prev, l_max=60.0)
        r_prev = st["r"]
        r1, q1, bits, weight = lit[p]
        np.testing.assert_allclose(st["r"], np.log(r1 / (1.0 - r1)), rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(st["post"], np.log(q1 / (1.0 - q1)), rtol=1e-10, atol=1e-10)
        np.testing.assert_array_equal(st["bits"], bits)
        np.testing.assert_array_equal(st["weight"], weight)


# --- invariants of the whole decoder ---------------------------------------------

@pytest.fixture(scope="module")
def n1008():
    code = I.small_code_n1008()
    cw = I.encode_ira(code, I.random_info(40, code.k, seed=21))
    return code, cw


def test_noiseless_codeword_decodes_in_zero_iterations(oracle_mod, n1008):
    code, cw = n1008
    lam = np.where(cw == 1, 40.0, -40.0)
    out = oracle_mod.decode(code, lam, 50)
    assert np.all(out["iters"] == 0) and np.all(out["ok"] == 1)
    np.testing.assert_array_equal(out["bits"], cw)


def test_all_zero_word_at_high_snr(oracle_mod, n1008):
    code, _ = n1008
    s2 = I.sigma2_from_ebn0(8.0, 0.5)
    lam = oracle_mod.gen_awgn(7, 0, 40, code.n, s2)
    out = oracle_mod.decode(code, lam, 50)
    assert out["bits"].sum() == 0 and np.all(out["ok"] == 1)


def test_codeword_sign_symmetry_is_exact(oracle_mod, n1008):
    """Flipping the LLR signs on a codeword c' flips exactly those decisions
    and negates those posteriors, with the same iteration counts."""
    code, cw = n1008
    s2 = I.sigma2_from_ebn0(1.5, 0.5)
    lam = I.gaussian_llr(np.zeros_like(cw), s2, seed=3).astype(np.float64)
    base = oracle_mod.decode(code, lam, 30)
    flip = oracle_mod.decode(code, lam * (1.0 - 2.0 * cw), 30)
    np.testing.assert_array_equal(flip["iters"], base["iters"])
    np.testing.assert_array_equal(flip["ok"], base["ok"])
    np.testing.assert_array_equal(flip["bits"], base["bits"] ^ cw)
    np.testing.assert_array_equal(flip["post"], base["post"] * (1.0 - 2.0 * cw))


def test_ok_iff_zero_syndrome_and_prefix_property(oracle_mod, n1008):
    code, cw = n1008
    s2 = I.sigma2_from_ebn0(1.25, 0.5)
    lam = I.gaussian_llr(cw, s2, seed=8).astype(np.float64)
    full = oracle_mod.decode(code, lam, 40)
    np.testing.assert_array_equal(full["ok"] == 1, oracle_mod.syndrome_weight(code, full["bits"]) == 0)
    for t in (0, 1, 3, 7):
        part = oracle_mod.decode(code, lam, t)
        early = full["iters"] <= t
        np.testing.assert_array_equal(part["iters"][early & (full["ok"] == 1)], full["iters"][early & (full["ok"] == 1)])
        assert np.all(part["iters"][~early] == t) and np.all(part["ok"][~early] == 0)
        # fixed mode with max_iter = t runs the same passes as early exit until t
        fixed = oracle_mod.decode(code, lam, t, early_exit=False)
        same = ~early
        np.testing.assert_array_equal(fixed["post"][same], part["post"][same])


def test_bp_frame_errors_not_below_ml(oracle_mod):
    """ML minimises the frame error rate, so FER_BP >= FER_ML (95% margin)."""
    code = I.ira_code(18, 9, {3: 1.0}, seed=2)
    words = oracle_mod.codewords_of(code)
    assert words.shape[0] == 2 ** 9
    s2 = I.sigma2_from_ebn0(1.0, 0.5)
    rng = np.random.default_rng(17)
    sent = words[rng.integers(0, words.shape[0], size=3000)]
    lam = I.gaussian_llr(sent, s2, seed=18).astype(np.float64)
    bp = oracle_mod.decode(code, lam, 50)
    ml = oracle_mod.ml_decode(words, lam)
    fer_bp = np.mean(np.any(bp["bits"] != sent, axis=1))
    fer_ml = np.mean(np.any(ml != sent, axis=1))
    margin = 1.96 * math.sqrt(fer_ml * (1 - fer_ml) / sent.shape[0] + fer_bp * (1 - fer_bp) / sent.shape[0])
    assert fer_bp >= fer_ml - margin
    assert fer_ml > 0.0


# --- channel generator (BER-simulator section; Philox from Salmon et al.) -----------

def test_philox_matches_numpy(oracle_mod):
    """numpy's Philox is Philox-4x64-10; it bumps the counter before each block."""
    for key0, key1, ctr0 in ((5, 0, 0), (2 ** 64 - 1, 12345, 77), (0x243F6A8885A308D3, 0x13198A2E03707344, 10 ** 12)):
        bg = np.random.Philox(key=np.array([key0, key1], dtype=np.uint64),
                              counter=np.array([ctr0, 0, 0, 0], dtype=np.uint64))
        want = bg.random_raw(4 * 64).reshape(64, 4)
        got = oracle_mod.philox_blocks(key0, key1, ctr0 + 1, 0, 64)
        np.testing.assert_array_equal(got, want)


def test_awgn_statistics(oracle_mod):
    n, f = 4000, 40
    s2 = I.sigma2_from_ebn0(1.0, 0.5)
    lam = oracle_mod.gen_awgn(99, 0, f, n, s2)
    z = (lam * s2 / 2.0 + 1.0) / math.sqrt(s2)  # back to the unit normal
    assert abs(z.mean()) < 4.0 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 0.02
    assert stats.kstest(z.ravel(), "norm").pvalue > 1e-3
    cw = np.ones((f, n), dtype=np.uint8)
    lam1 = oracle_mod.gen_awgn(99, 0, f, n, s2, cw)
    np.testing.assert_allclose(lam1 - lam, 4.0 / s2, rtol=1e-12)


def test_awgn_frames_are_independent_of_batching(oracle_mod):
    s2 = 0.7
    whole = oracle_mod.gen_awgn(3, 100, 10, 37, s2)
    part = oracle_mod.gen_awgn(3, 104, 3, 37, s2)
    np.testing.assert_array_equal(whole[4:7], part)


def test_paper_sweep_stand_in_codes_have_four_edges_per_bit(oracle_mod):
    """The Table 3 stand-ins: rate 1/2 and E = 4n - 1 (the paper lists 4n)."""
    from paper_1609_01567_gb300 import sweep
    for n in (256, 512, 4096):
        code = sweep.stand_in_code(n)
        assert code.n == n and code.m == n // 2 and code.n_edges == 4 * n - 1
        cw = I.encode_ira(code, I.random_info(3, code.k, seed=n))
        assert np.all(oracle_mod.syndrome_weight(code, cw) == 0)
    assert sorted(sweep.PAPER_TABLE3_SECONDS) == [2 ** p for p in range(8, 19)]


# --- min-sum family (a derived algorithm the paper names) -------------------------

def max_log_parity(lam):
    """Brute-force max-log LLR of each bit of one parity check: over the
    other bits' configurations x with the right parity, max sum x*lambda for
    c_j = 1 minus the same for c_j = 0."""
    import itertools
    f, d = lam.shape
    out = np.zeros_like(lam)
    for j in range(d):
        others = [t for t in range(d) if t != j]
        best = {0: np.full(f, -np.inf), 1: np.full(f, -np.inf)}
        for x in itertools.product((0, 1), repeat=d - 1):
            par = sum(x) % 2  # c_j must equal the parity of the others
            score = sum(lam[:, t] * xi for t, xi in zip(others, x))
            best[par] = np.maximum(best[par], score)
        out[:, j] = best[1] - best[0]
    return out


@pytest.mark.parametrize("d", [2, 3, 4, 6])
def test_min_sum_is_max_log_on_one_check(oracle_mod, d):
    code = I.coo_code(1, d, [0] * d, list(range(d)))
    lam = np.random.default_rng(d).normal(0.0, 3.0, size=(25, d))
    out = oracle_mod.decode(code, lam, 0, early_exit=False, l_max=60.0, rule="min_sum")
    np.testing.assert_allclose(out["post"] - lam, max_log_parity(lam), rtol=1e-12, atol=1e-12)


def test_min_sum_variants_and_bounds(oracle_mod):
    """Degree-2 checks: min-sum equals sum-product. Normalised and offset
    variants scale and shift the plain messages; min-sum magnitudes never
    fall below the sum-product ones on the first pass."""
    code2 = I.coo_code(1, 2, [0, 0], [0, 1])
    lam2 = np.random.default_rng(1).normal(0.0, 4.0, size=(30, 2))
    sp = oracle_mod.decode(code2, lam2, 0, early_exit=False)
    ms = oracle_mod.decode(code2, lam2, 0, early_exit=False, rule="min_sum")
    np.testing.assert_allclose(ms["post"], sp["post"], rtol=1e-12, atol=1e-9)
    code = I.small_code_n1008()
    lam = I.gaussian_llr(np.zeros((6, code.n), np.uint8), I.sigma2_from_ebn0(1.0, 0.5), seed=2).astype(np.float64)
    plain = oracle_mod.sp_pass(code, lam, rule="min_sum")["r"]
    norm = oracle_mod.sp_pass(code, lam, rule="min_sum", alpha=0.75)["r"]
    off = oracle_mod.sp_pass(code, lam, rule="min_sum", beta=0.5)["r"]
    np.testing.assert_allclose(norm, 0.75 * plain, rtol=1e-14)
    np.testing.assert_allclose(off, np.sign(plain) * np.maximum(np.abs(plain) - 0.5, 0.0), rtol=1e-14, atol=1e-15)
    exact = oracle_mod.sp_pass(code, lam)["r"]
    assert np.all(np.abs(plain) >= np.abs(exact) - 1e-12)


def _scaled_max_log(lam, alpha, beta):
    ml = max_log_parity(lam)
    return np.sign(ml) * np.maximum(alpha * np.abs(ml) - beta, 0.0)


def test_adaptive_min_sum_scales_each_check_by_its_own_degree(oracle_mod):
    """Two disjoint checks of degrees 3 and 5: after the first check pass each
    bit's extrinsic LLR is its check's brute-force max-log value with that
    degree's scale and offset. The neighbouring table entries (degrees 2, 4,
    6) hold other values, so reading the table at d - 1, d + 1 or at a
    variable's degree fails."""
    rows = [0, 0, 0] + [1] * 5
    cols = list(range(8))
    code = I.coo_code(2, 8, rows, cols)
    alpha = [9.0, 9.0, 0.3, 0.6, 0.45, 0.8, 0.2]
    beta = [0.0, 0.0, 0.7, 0.1, 0.5, 0.25, 1.3]
    lam = np.random.default_rng(7).normal(0.0, 3.0, size=(40, 8))
    out = oracle_mod.decode(code, lam, 0, early_exit=False, l_max=60.0, rule="min_sum_adaptive",
                            alpha_by_degree=alpha, beta_by_degree=beta)
    ext = out["post"] - lam
    np.testing.assert_allclose(ext[:, :3], _scaled_max_log(lam[:, :3], 0.6, 0.1), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ext[:, 3:], _scaled_max_log(lam[:, 3:], 0.8, 0.25), rtol=1e-12, atol=1e-12)


def test_adaptive_min_sum_degrees_past_the_table_take_its_last_entry(oracle_mod):
    code = I.coo_code(1, 6, [0] * 6, list(range(6)))
    lam = np.random.default_rng(8).normal(0.0, 3.0, size=(30, 6))
    out = oracle_mod.decode(code, lam, 0, early_exit=False, l_max=60.0, rule="min_sum_adaptive",
                            alpha_by_degree=[1.0, 1.0, 0.5, 0.7], beta_by_degree=[0.0, 0.0, 0.0, 0.4])
    np.testing.assert_allclose(out["post"] - lam, _scaled_max_log(lam, 0.7, 0.4), rtol=1e-12, atol=1e-12)


def test_adaptive_min_sum_with_one_value_for_every_degree_is_the_plain_variant(oracle_mod, n1008):
    """A table holding one (alpha, beta) for every degree reduces the adaptive
    rule to the normalised/offset rule, pass for pass and bit for bit."""
    code, cw = n1008
    lam = I.gaussian_llr(cw[:6], I.sigma2_from_ebn0(1.5, 0.5), seed=9).astype(np.float64)
    fixed = oracle_mod.decode(code, lam, 12, early_exit=False, rule="min_sum", alpha=0.75, beta=0.25)
    adapt = oracle_mod.decode(code, lam, 12, early_exit=False, rule="min_sum_adaptive",
                              alpha_by_degree=[0.75] * 3, beta_by_degree=[0.25] * 3)
    np.testing.assert_array_equal(adapt["post"], fixed["post"])
    np.testing.assert_array_equal(adapt["iters"], fixed["iters"])


@pytest.mark.parametrize("alpha,beta", [([], []), ([0.5, 0.0], [0.0, 0.0]), ([0.5, 0.5], [0.0, -0.1]),
                                        ([0.5, np.inf], [0.0, 0.0]), ([0.5, 0.5], [0.0, np.nan])])
def test_adaptive_min_sum_rejects_bad_tables(oracle_mod, alpha, beta):
    code = I.coo_code(1, 3, [0, 0, 0], [0, 1, 2])
    with pytest.raises(ValueError):
        oracle_mod.decode(code, np.zeros((1, 3)), 1, rule="min_sum_adaptive", alpha_by_degree=alpha,
                          beta_by_degree=beta)


# --- quantised message storage (int8: step 20/127, |k| <= 127) ----------------

def test_quantised_messages_lie_on_the_int8_lattice_and_round_to_nearest(oracle_mod, n1008):
    """Stored messages are k * 20/127 with |k| <= 127, within half a step of
    the unrounded messages computed from the same inputs, and the APP sums the
    stored (not the unrounded) messages."""
    code, cw = n1008
    step = 20.0 / 127.0
    lam = I.gaussian_llr(cw[:8], I.sigma2_from_ebn0(1.5, 0.5), seed=5).astype(np.float64)
    q0 = oracle_mod.sp_pass(code, lam, msg="i8")
    prev = q0["r"]
    for r_prev in (None, prev):
        exact = oracle_mod.sp_pass(code, lam, r_prev)
        quant = oracle_mod.sp_pass(code, lam, r_prev, msg="i8")
        k = quant["r"] / step
        np.testing.assert_allclose(k, np.round(k), atol=1e-9)
        assert np.abs(k).max() <= 127 + 1e-9
        assert np.abs(quant["r"] - exact["r"]).max() <= step / 2 + 1e-12
        v = oracle_mod.address_iterators(code)["v"]
        app = lam.copy()
        for f in range(lam.shape[0]):
            np.add.at(app[f], v, quant["r"][f])
        np.testing.assert_allclose(quant["post"], app, rtol=1e-12, atol=1e-12)
        np.testing.assert_array_equal(quant["bits"], (app > 0).astype(np.uint8))
    # a saturated message is stored at the top level: a degree-2 check passes
    # its other input clamped to L_MAX = 20 = 127 steps
    code2 = I.coo_code(1, 2, [0, 0], [0, 1])
    out = oracle_mod.sp_pass(code2, np.array([[35.0, -3.0]]), msg="i8")
    np.testing.assert_allclose(out["r"][0], [np.round(-3.0 / step) * step, 127 * step], atol=1e-12)


def test_fine_quantisation_reduces_to_unrounded_decoder(oracle_mod, n1008):
    code, cw = n1008
    lam = I.gaussian_llr(cw[:10], I.sigma2_from_ebn0(1.25, 0.5), seed=6).astype(np.float64)
    exact = oracle_mod.decode(code, lam, 25)
    fine = oracle_mod.decode(code, lam, 25, msg=(1e-8, 2 ** 31 - 1))  # top level 21.5 > L_MAX
    np.testing.assert_array_equal(fine["iters"], exact["iters"])
    np.testing.assert_array_equal(fine["bits"], exact["bits"])
    np.testing.assert_allclose(fine["post"], exact["post"], rtol=0, atol=1e-6)


def test_quantised_decoder_keeps_codeword_symmetry(oracle_mod, n1008):
    """Rounding to the nearest level (ties to even) is odd-symmetric, so the
    int8 decoder keeps the exact codeword sign symmetry."""
    code, cw = n1008
    lam = I.gaussian_llr(np.zeros_like(cw), I.sigma2_from_ebn0(1.5, 0.5), seed=3).astype(np.float64)
    base = oracle_mod.decode(code, lam, 30, msg="i8")
    flip = oracle_mod.decode(code, lam * (1.0 - 2.0 * cw), 30, msg="i8")
    np.testing.assert_array_equal(flip["iters"], base["iters"])
    np.testing.assert_array_equal(flip["bits"], base["bits"] ^ cw)
    np.testing.assert_array_equal(flip["post"], base["post"] * (1.0 - 2.0 * cw))
    assert base["ok"].mean() > 0.5


# --- 16-bit floating-point message storage (binary16, bfloat16) ---------------------

def _nearest_by_patterns(x, fmt):
    """The value of ``fmt`` nearest to x > 0 found by enumerating bit patterns
    around x (ties to the even pattern): binary16 patterns through numpy's
    float16 type, bfloat16 patterns as float32 patterns with 16 zero low bits."""
    import struct
    if fmt == "f16":
        b0 = int(np.array([x], dtype=np.float64).astype(np.float16).view(np.uint16)[0])
        cands = [(float(np.array([b], dtype=np.uint16).view(np.float16)[0]), b) for b in range(max(b0 - 3, 0), b0 + 4)
                 if b < 0x7c00]
    else:
        b0 = struct.unpack("<I", struct.pack("<f", float(np.float32(x))))[0] >> 16
        cands = [(struct.unpack("<f", struct.pack("<I", b << 16))[0], b) for b in range(max(b0 - 3, 0), b0 + 4)]
    best = min(abs(x - v) for v, _ in cands)
    ties = [(v, b) for v, b in cands if abs(x - v) == best]
    return next(v for v, b in ties if b % 2 == 0) if len(ties) > 1 else ties[0][0]


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_16_bit_storage_rounds_to_nearest_even(oracle_mod, fmt):
    """The oracle's binary16/bfloat16 rounding against a brute-force search
    over bit patterns: random magnitudes from 1e-9 (binary16 subnormals and
    underflow) to 30, exact midpoints between neighbouring values (ties go to
    the even pattern), representable values (unchanged), zero and odd
    symmetry; binary16 also against numpy's float16 conversion."""
    rng = np.random.default_rng(16)
    xs = list(np.exp(rng.uniform(np.log(1e-9), np.log(30.0), 3000)))
    for x in xs[:200]:  # a value, its successor (next bit pattern) and their midpoint, a tie
        lo = _nearest_by_patterns(x, fmt)
        hi = _next_up(lo, fmt)
        xs += [lo, hi, (lo + hi) / 2.0]
    ties = 0
    for x in xs:
        want = _nearest_by_patterns(x, fmt)
        got = oracle_mod.store(x, fmt)
        ties += abs(x - _next_up(got, fmt)) == abs(x - got) or (got > 0 and abs(x - got) == abs(x - _next_down(got, fmt)))
        assert got == want, (fmt, x, got, want)
        assert oracle_mod.store(-x, fmt) == -got
        if fmt == "f16":
            assert got == float(np.float16(x)), (x, got)
    assert oracle_mod.store(0.0, fmt) == 0.0
    assert ties >= 150, ties  # the midpoints are exact ties


def _pattern(v, fmt):
    import struct
    if fmt == "f16":
        return int(np.array([v], dtype=np.float64).astype(np.float16).view(np.uint16)[0])
    return struct.unpack("<I", struct.pack("<f", float(np.float32(v))))[0] >> 16


def _value(b, fmt):
    import struct
    if fmt == "f16":
        return float(np.array([b], dtype=np.uint16).view(np.float16)[0])
    return struct.unpack("<f", struct.pack("<I", b << 16))[0]


def _next_up(v, fmt):
    return _value(_pattern(v, fmt) + 1, fmt)


def _next_down(v, fmt):
    return _value(_pattern(v, fmt) - 1, fmt)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_16_bit_stored_messages_and_posteriors(oracle_mod, n1008, fmt):
    """Stored messages are values of the format, each the nearest one to the
    unrounded message from the same inputs; the APP sums the stored messages;
    the decoder keeps the exact codeword sign symmetry (rounding to nearest
    even is odd-symmetric)."""
    code, cw = n1008
    lam = I.gaussian_llr(cw[:8], I.sigma2_from_ebn0(1.5, 0.5), seed=5).astype(np.float64)
    prev = oracle_mod.sp_pass(code, lam, msg=fmt)["r"]
    v = oracle_mod.address_iterators(code)["v"]
    for r_prev in (None, prev):
        exact = oracle_mod.sp_pass(code, lam, r_prev)
        stored = oracle_mod.sp_pass(code, lam, r_prev, msg=fmt)
        r = stored["r"]
        if fmt == "f16":
            np.testing.assert_array_equal(r.astype(np.float16).astype(np.float64), r)
        else:
            bits = r.astype(np.float32).view(np.uint32)
            np.testing.assert_array_equal(r.astype(np.float32).astype(np.float64), r)
            assert not np.any(bits & 0xFFFF)
        sample = np.random.default_rng(1).choice(r.size, 300, replace=False)
        for i in sample:
            u = exact["r"].flat[i]
            assert r.flat[i] == np.sign(u) * _nearest_by_patterns(abs(u), fmt) or u == 0.0
        app = lam.copy()
        for f in range(lam.shape[0]):
            np.add.at(app[f], v, r[f])
        np.testing.assert_allclose(stored["post"], app, rtol=1e-12, atol=1e-12)
    lam0 = I.gaussian_llr(np.zeros_like(cw), I.sigma2_from_ebn0(1.5, 0.5), seed=3).astype(np.float64)
    base = oracle_mod.decode(code, lam0, 30, msg=fmt)
    flip = oracle_mod.decode(code, lam0 * (1.0 - 2.0 * cw), 30, msg=fmt)
    np.testing.assert_array_equal(flip["iters"], base["iters"])
    np.testing.assert_array_equal(flip["bits"], base["bits"] ^ cw)
    np.testing.assert_array_equal(flip["post"], base["post"] * (1.0 - 2.0 * cw))


# --- tabulated phi (rule "sp_table") ------------------------------------------------

def test_tabulated_phi_is_the_chord_of_a_convex_function(oracle_mod):
    """phi is convex on (0, inf), so each chord lies on or above it and meets
    it at the bucket edges; with 64 buckets per octave the chord stays within
    a small relative distance. Edges are floats whose bits are key << 17."""
    import struct
    rng = np.random.default_rng(0)
    xs = np.concatenate([np.exp(rng.uniform(np.log(4e-9), np.log(22.0), 4000)), [1e-8, 0.5, 1.0, 2.0, 20.0]])
    worst_abs = worst_rel_small = worst_rel = 0.0
    for x in xs:
        t, p = oracle_mod.phi_chord(x), oracle_mod.phi(x)
        assert t >= p * (1 - 1e-12)
        worst_abs = max(worst_abs, t - p)
        worst_rel = max(worst_rel, (t - p) / p)
        if x <= 1.0:
            worst_rel_small = max(worst_rel_small, (t - p) / p)
    # chord error ~ (bucket width)^2 / 8 * phi'': tiny in absolute terms, and
    # relative to phi at most ~(x / 64)^2 / 8 where phi ~ 2 e^-x
    assert worst_abs < 5e-5 and worst_rel_small < 2e-4 and worst_rel < 1e-2, (worst_abs, worst_rel_small, worst_rel)
    for key in (95 << 6, (120 << 6) + 17, (127 << 6) + 5, (131 << 6) + 63):
        e = struct.unpack("<f", struct.pack("<I", key << 17))[0]
        assert abs(oracle_mod.phi_chord(e) - oracle_mod.phi(e)) <= 1e-12 * oracle_mod.phi(e)
        # continuous across the edge
        assert abs(oracle_mod.phi_chord(e * (1 - 1e-9)) - oracle_mod.phi_chord(e)) <= 1e-6 * oracle_mod.phi(e)


def test_tabulated_rule_tracks_exact_sum_product(oracle_mod, n1008):
    """One check: the tabulated rule is phi_T(sum phi_T); on the n = 1008 code
    it decodes like exact sum-product (same decisions on converged frames,
    posteriors within a few parts per thousand on the first pass)."""
    code1 = I.coo_code(1, 4, [0] * 4, [0, 1, 2, 3])
    lam = np.array([[0.7, -1.9, 3.3, 0.2]])
    out = oracle_mod.sp_pass(code1, lam, rule="sp_table")["r"][0]
    mags = [oracle_mod.phi_chord(abs(v)) for v in lam[0]]
    for k in range(4):
        want = oracle_mod.phi_chord(sum(mags) - mags[k])
        others = sum(1 for j in range(4) if j != k and lam[0, j] > 0)
        assert abs(abs(out[k]) - want) < 1e-12 and (out[k] > 0) == (others % 2 == 1)
    code, cw = n1008
    llr = I.gaussian_llr(cw[:30], I.sigma2_from_ebn0(2.0, 0.5), seed=12).astype(np.float64)
    ex = oracle_mod.sp_pass(code, llr)
    tb = oracle_mod.sp_pass(code, llr, rule="sp_table")
    assert np.abs(tb["r"] - ex["r"]).max() < 5e-3 * (1 + np.abs(ex["r"]).max())
    a = oracle_mod.decode(code, llr, 50)
    b = oracle_mod.decode(code, llr, 50, rule="sp_table")
    both = (a["ok"] == 1) & (b["ok"] == 1)
    assert (a["iters"] == b["iters"]).mean() >= 0.9 and abs(int(a["ok"].sum()) - int(b["ok"].sum())) <= 1
    np.testing.assert_array_equal(a["bits"][both], b["bits"][both])
