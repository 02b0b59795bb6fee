"""Device information bits, the IRA encoder, lifted (QC) codes and
random-codeword simulation, against the oracle.

Encoder: the staircase makes H2 invertible, so a word is THE codeword of its
information part iff its first k bits are that part and its syndrome is zero;
both are checked with the oracle's syndrome, and the words are also compared
with the host encoder of the input generator.
"""
import numpy as np
import pytest

from paper_1609_01567_gb300 import ber
from paper_1609_01567_gb300 import inputs as I
from tests.parity import close, gf2_information_positions, near_zero_frames

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


def expected_bits(oracle_mod, seed, offset, F, k):
    """Bit j of frame f: bit j % 64 of word (j % 256) // 64 of the Philox
    block (key (seed, 1), counter (j // 256, offset + f))."""
    nb = (k + 255) // 256
    out = np.zeros((F, k), dtype=np.uint8)
    q = np.arange(256)
    for f in range(F):
        blk = oracle_mod.philox_blocks(seed, 1, 0, offset + f, nb)
        bits = (blk[:, q // 64] >> (q % 64).astype(np.uint64)) & np.uint64(1)
        out[f] = bits.reshape(-1)[:k].astype(np.uint8)
    return out


@pytest.mark.parametrize("F,k,offset", [(1, 7, 0), (5, 1000, 3), (33, 257, 11), (3, 32400, 1 << 33)])
def test_gen_bits_match_philox(ldpc, oracle_mod, F, k, offset):
    got = ldpc.ldpc_gen_bits(77, offset, F, k).cpu().numpy()
    np.testing.assert_array_equal(got, expected_bits(oracle_mod, 77, offset, F, k))


def test_gen_bits_unaligned_rows(ldpc, oracle_mod):
    """Rows that start off an 8-byte boundary take the byte-store path."""
    buf = torch.zeros(4 * 77 + 1, dtype=torch.uint8, device="cuda")
    out = buf[1:].view(4, 77)
    ldpc.ldpc_gen_bits(5, 0, 4, 77, out=out)
    np.testing.assert_array_equal(out.cpu().numpy(), expected_bits(oracle_mod, 5, 0, 4, 77))
    assert buf[0].item() == 0


@pytest.mark.parametrize("which,F", [("n1008", 1), ("n1008", 31), ("n1008", 33), ("n1008", 100), ("n64800", 64)])
def test_ira_encoder(ldpc, oracle_mod, which, F):
    code = I.small_code_n1008() if which == "n1008" else I.large_code_n64800()
    h = ldpc.code_from_inputs(code)
    info = I.random_info(F, code.k, seed=F)
    cw = ldpc.ldpc_encode_ira(h, torch.from_numpy(info).cuda()).cpu().numpy()
    np.testing.assert_array_equal(cw[:, :code.k], info)
    assert np.all(oracle_mod.syndrome_weight(code, cw) == 0)
    np.testing.assert_array_equal(cw, I.encode_ira(code, info))


def test_ira_encoder_mixed_codes(ldpc, oracle_mod):
    for code in I.mixed_codes():
        h = ldpc.code_from_inputs(code)
        info = I.random_info(40, code.k, seed=code.n)
        cw = ldpc.ldpc_encode_ira(h, torch.from_numpy(info).cuda()).cpu().numpy()
        np.testing.assert_array_equal(cw[:, :code.k], info)
        assert np.all(oracle_mod.syndrome_weight(code, cw) == 0), code.name


def test_encoder_refuses_non_ira_code(ldpc):
    code, ent = I.qc_stand_in_code(256)
    h = ldpc.ldpc_code_create_qc(4, 8, 32, ent)
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_encode_ira(h, torch.zeros((2, 128), dtype=torch.uint8, device="cuda"))
    assert e.value.status == -1 and "staircase" in str(e.value)


def test_qc_code_decodes_like_the_oracle(ldpc, oracle_mod):
    code, ent = I.qc_stand_in_code(2048)
    h = ldpc.ldpc_code_create_qc(4, 8, 2048 // 8, ent)
    lam = I.gaussian_llr(np.zeros((300, code.n), np.uint8), I.sigma2_from_ebn0(2.5, 0.5), seed=31)
    out = ldpc.ldpc_decode(h, torch.from_numpy(np.ascontiguousarray(lam, dtype=np.float32)).cuda(), 30)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    ref = oracle_mod.decode(code, lam.astype(np.float64), 30, n_threads=8)
    same = (got["bits"] == ref["bits"]).all(axis=1) & (got["iters"] == ref["iters"]) & (got["ok"] == ref["ok"])
    exempt = near_zero_frames(ref["post"])
    assert np.all(same | exempt), np.flatnonzero(~same & ~exempt)[:10]
    short = ref["iters"] <= 15
    assert close(got["post"], ref["post"]).all(axis=1)[short & ~exempt].all()
    assert (ref["ok"] == 1).mean() > 0.5


def test_random_codeword_simulation(ldpc, oracle_mod):
    """Random codewords made on the device decode as well as the all-zero
    word (linearity and the decoder's symmetry), and the counted errors are
    relative to the transmitted words: at high SNR nothing is miscounted."""
    code = I.small_code_n1008()
    h = ldpc.code_from_inputs(code)
    z = ber.simulate(h, code, 1.5, 4000, batch=1000, seed=3)
    r = ber.simulate(h, code, 1.5, 4000, batch=1000, seed=3, codewords="random")
    lo_z, hi_z = ber.wilson(z.frame_errors, 4000)
    lo_r, hi_r = ber.wilson(r.frame_errors, 4000)
    assert lo_z <= hi_r and lo_r <= hi_z, (z, r)
    hi = ber.simulate(h, code, 6.0, 2000, batch=1000, seed=4, codewords="random")
    assert hi.frame_errors == 0 and hi.bit_errors == 0 and hi.unsatisfied == 0
    # the transmitted words themselves: what the device made, as the oracle sees it
    info = ldpc.ldpc_gen_bits(3, 0, 50, code.k)
    cw = ldpc.ldpc_encode_ira(h, info).cpu().numpy()
    assert np.all(oracle_mod.syndrome_weight(code, cw) == 0)
    np.testing.assert_array_equal(cw[:, :code.k], expected_bits(oracle_mod, 3, 0, 50, code.k))


def test_dense_encoder_on_a_lifted_code(ldpc, oracle_mod):
    """The dense systematic encoder on a lifted (4, 8) code without a
    staircase: every word satisfies H c = 0 (the oracle's syndrome) and holds
    its information bits at the information positions that an independent
    GF(2) basis computation finds (columns in the span of the columns to
    their right); together these fix the codeword."""
    code, ent = I.qc_stand_in_code(512)
    h = ldpc.ldpc_code_create_qc(4, 8, 64, ent)
    pos, rank = gf2_information_positions(code.m, code.n, code.rows, code.cols)
    k = ldpc.ldpc_code_build_encoder(h)
    assert k == len(pos) == code.n - rank
    for F in (1, 33, 70):
        info = I.random_info(F, k, seed=F)
        cw = ldpc.ldpc_encode(h, torch.from_numpy(info).cuda()).cpu().numpy()
        np.testing.assert_array_equal(cw[:, pos], info)
        assert np.all(oracle_mod.syndrome_weight(code, cw) == 0), F


def test_dense_encoder_equals_the_ira_encoder(ldpc):
    """On an IRA code the dense encoder's parity positions are the staircase
    columns, so its words are the IRA encoder's, bit for bit."""
    for code in (I.small_code_n1008(), I.mixed_codes()[3]):
        h = ldpc.code_from_inputs(code)
        assert ldpc.ldpc_code_build_encoder(h) == code.k
        info = torch.from_numpy(I.random_info(45, code.k, seed=9)).cuda()
        np.testing.assert_array_equal(ldpc.ldpc_encode(h, info).cpu().numpy(),
                                      ldpc.ldpc_encode_ira(h, info).cpu().numpy(), err_msg=code.name)


def test_random_codewords_of_a_lifted_code(ldpc, oracle_mod):
    """Random codewords of a lifted code (dense encoder) decode as well as the
    all-zero word, and at high SNR nothing is miscounted."""
    code, ent = I.qc_stand_in_code(2048)
    h = ldpc.ldpc_code_create_qc(4, 8, 256, ent)
    z = ber.simulate(h, code, 2.2, 3000, batch=1000, seed=5)
    r = ber.simulate(h, code, 2.2, 3000, batch=1000, seed=5, codewords="random")
    lo_z, hi_z = ber.wilson(z.frame_errors, 3000)
    lo_r, hi_r = ber.wilson(r.frame_errors, 3000)
    assert lo_z <= hi_r and lo_r <= hi_z, (z, r)
    hi = ber.simulate(h, code, 6.0, 1000, batch=1000, seed=6, codewords="random")
    assert hi.frame_errors == 0 and hi.bit_errors == 0 and hi.unsatisfied == 0
    k = ldpc.ldpc_code_build_encoder(h)
    cw = ldpc.ldpc_encode(h, ldpc.ldpc_gen_bits(6, 0, 40, k)).cpu().numpy()
    assert np.all(oracle_mod.syndrome_weight(code, cw) == 0) and cw.any()
