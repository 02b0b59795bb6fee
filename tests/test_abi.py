"""The C ABI on the CPU: symbols, host tables, argument errors (no GPU work).

Codes are created host-only (device -1), which builds the tables without
touching a GPU; decoding such a code must refuse with LDPC_ENODEV.
"""
import ctypes
import re
import subprocess
from pathlib import Path

import numpy as np
import pytest

from paper_1609_01567_gb300 import build as lib_build
from paper_1609_01567_gb300 import inputs as I
from tests.paper_tables import table
from tests.parity import gf2_information_positions

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def ldpc():
    lib_build.build()
    from paper_1609_01567_gb300 import ldpc as mod
    return mod


def declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(ldpc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(ldpc):
    names = declared_functions()
    assert {"ldpc_code_create", "ldpc_decode", "ldpc_gen_awgn"} <= names
    out = subprocess.run(["nm", "-D", "--defined-only", str(lib_build.library_path())], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = names - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    assert set(ldpc.EXPORTS) == names
    lib = ldpc.library()
    for n in names:
        getattr(lib, n)
    assert "sm_103a" in ldpc.ldpc_version()


def test_host_tables_reproduce_tables_1_and_2(ldpc):
    code = I.code_14_7()
    h = ldpc.ldpc_code_create(code.m, code.n, code.rows, code.cols, device=-1)
    got = ldpc.ldpc_code_tables(h)
    for number in (1, 2):
        for name, want in table(number).items():
            if name == "e":
                continue
            np.testing.assert_array_equal(got[name], want, err_msg=f"Table {number} array {name}")


def test_edge_ids_follow_a_stable_sort_by_column(ldpc):
    """Shuffling the COO and reading the tables back gives the same graph,
    with edge ids ordered by (column, position in the COO)."""
    code = I.small_code_n1008()
    rng = np.random.default_rng(1)
    perm = rng.permutation(code.n_edges)
    rows, cols = code.rows[perm], code.cols[perm]
    h = ldpc.ldpc_code_create(code.m, code.n, rows, cols, device=-1)
    t = ldpc.ldpc_code_tables(h)
    order = np.argsort(cols, kind="stable")
    np.testing.assert_array_equal(t["v"], cols[order])
    np.testing.assert_array_equal(t["c"], rows[order])
    np.testing.assert_array_equal(t["ebar"], np.argsort(t["c"], kind="stable"))
    np.testing.assert_array_equal(t["vbar"], t["v"][t["ebar"]])


def test_code_info_and_degree_bins(ldpc):
    code = I.large_code_n64800()
    h = ldpc.ldpc_code_create(code.m, code.n, code.rows, code.cols, device=-1)
    info = ldpc.ldpc_code_info(h)
    assert info["m"] == 32400 and info["n"] == 64800 and info["n_edges"] == 194399
    assert info["max_check_degree"] == 6 and info["max_var_degree"] == 8
    assert info["check_bin_count"] == [0, 32400, 0, 0, 0, 0]
    assert info["device"] == -1
    big = I.ira_code(8192, 6144, {3: 0.7, 4: 0.3}, seed=3, var_degree_overrides={0: 64},
                     check_h1_overrides={5: 94})
    hb = ldpc.ldpc_code_create(big.m, big.n, big.rows, big.cols, device=-1)
    ib = ldpc.ldpc_code_info(hb)
    assert ib["max_check_degree"] == 96 and ib["max_var_degree"] == 64
    assert ib["check_bin_count"][5] == 1


def test_argument_errors(ldpc):
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_code_create(2, 2, [0, 0], [1, 1], device=-1)
    assert e.value.status == -2 and "more than once" in str(e.value)
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_code_create(2, 2, [0, 2], [1, 1], device=-1)
    assert e.value.status == -1
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_code_create(-1, 2, [], [], device=-1)
    assert e.value.status == -1
    empty = ldpc.ldpc_code_create(3, 4, [], [], device=-1)
    assert ldpc.ldpc_code_info(empty)["n_edges"] == 0
    lib = ldpc.library()
    h = ldpc.ldpc_code_create(1, 2, [0, 0], [0, 1], device=-1)
    st = lib.ldpc_decode(h.handle, None, 1, 5, None, None, None, None, None, None)
    assert st == -7
    assert lib.ldpc_gen_awgn(1, 0, 1, 4, ctypes.c_float(0.0), None, None, None) == -1
    assert lib.ldpc_gen_awgn(1, 0, -1, 4, ctypes.c_float(1.0), None, None, None) == -1
    assert lib.ldpc_philox4x64_10(0, 0, 0, 0, -1, None, None) == -1
    # the entry points added beside the decoder refuse the same way
    assert lib.ldpc_decode_host_stream(h.handle, 1, None, 1, 5, None, None, None, None, None) == -7
    assert lib.ldpc_encode_ira(h.handle, None, 1, None, None) == -7
    assert lib.ldpc_gen_bits(1, 0, -1, 4, None, None) == -1
    assert lib.ldpc_gen_bits(1, -1, 1, 4, None, None) == -1
    assert lib.ldpc_gen_bits(1, 0, 0, 4, None, None) == 0  # nothing to do


def test_qc_lifting_matches_the_expanded_matrix(ldpc, oracle_mod):
    """Lifting in the library gives the Table 1-2 arrays of the explicitly
    expanded H (the oracle's address iterators), including parallel
    protograph edges (two shifts at one block)."""
    Z = 7
    entries = [(0, 0, 0), (0, 1, 3), (0, 1, 5), (1, 0, 6), (1, 2, 1), (2, 2, 0), (2, 3, 4), (1, 3, 2)]
    code = I.qc_code(3, 4, Z, entries)
    h = ldpc.ldpc_code_create_qc(3, 4, Z, entries, device=-1)
    got = ldpc.ldpc_code_tables(h)
    want = oracle_mod.address_iterators(code)
    for name in ("v", "c", "t", "s", "u", "ebar", "vbar", "cbar", "tbar", "sbar", "ubar"):
        np.testing.assert_array_equal(got[name], want[name], err_msg=name)
    dense = np.zeros((3 * Z, 4 * Z), dtype=np.int64)
    np.add.at(dense, (code.rows, code.cols), 1)
    assert dense.max() == 1 and dense.sum() == len(entries) * Z
    # block (0, 1) holds P^3 + P^5: row t has ones at columns 7 + (t + 3) % 7 and 7 + (t + 5) % 7
    for t in range(Z):
        assert set(np.flatnonzero(dense[t, Z:2 * Z])) == {(t + 3) % Z, (t + 5) % Z}
    info = ldpc.ldpc_code_info(h)
    assert info["ira_k"] == -1 and info["m"] == 3 * Z and info["n"] == 4 * Z


def test_qc_lifting_errors(ldpc):
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_code_create_qc(2, 2, 4, [(0, 0, 4)], device=-1)
    assert e.value.status == -1
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_code_create_qc(2, 2, 4, [(2, 0, 1)], device=-1)
    assert e.value.status == -1
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_code_create_qc(2, 2, 4, [(0, 0, 1), (1, 1, 0), (0, 0, 1)], device=-1)
    assert "repeats" in str(e.value)
    with pytest.raises(ldpc.LdpcError):
        ldpc.ldpc_code_create_qc(2, 2, 0, [], device=-1)


def test_ira_form_is_detected(ldpc):
    for code in (I.small_code_n1008(), I.mixed_codes()[4]):
        h = ldpc.ldpc_code_create(code.m, code.n, code.rows, code.cols, device=-1)
        assert ldpc.ldpc_code_info(h)["ira_k"] == code.k == code.n - code.m, code.name
    # swapping the last staircase column with information column 0 leaves IRA form
    code = I.small_code_n1008()
    last = code.n - 1
    cols = np.where(code.cols == last, 0, np.where(code.cols == 0, last, code.cols))
    h = ldpc.ldpc_code_create(code.m, code.n, code.rows, cols, device=-1)
    assert ldpc.ldpc_code_info(h)["ira_k"] == -1


def test_rule_table_validation(ldpc):
    code = I.code_14_7()
    h = ldpc.ldpc_code_create(code.m, code.n, code.rows, code.cols, device=-1)
    for alpha, beta in (([], None), ([0.5, 0.0], None), ([0.5, -1.0], None), ([0.5], [-0.1]),
                        ([float("inf")], None), ([0.5], [float("nan")])):
        with pytest.raises(ldpc.LdpcError) as e:
            ldpc.ldpc_code_set_rule_table(h, alpha, beta)
        assert e.value.status == -1 and ("entry" in str(e.value) or "n_degrees" in str(e.value)), str(e.value)
    with pytest.raises(ldpc.LdpcError) as e:  # a valid table needs device tables to land in
        ldpc.ldpc_code_set_rule_table(h, [0.8, 0.7], [0.0, 0.1])
    assert "host-only" in str(e.value)
    with pytest.raises(ValueError):
        ldpc.ldpc_code_set_rule_table(h, [0.8, 0.7], [0.1])


def test_debug_giveup_hook_validation(ldpc):
    code = I.code_14_7()
    h = ldpc.ldpc_code_create(code.m, code.n, code.rows, code.cols, device=-1)
    ldpc.ldpc_debug_giveup(h, 0)
    ldpc.ldpc_debug_giveup(h, -1)
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_debug_giveup(h, -2)
    assert e.value.status == -1


def test_dense_encoder_rank_and_positions(ldpc):
    """ldpc_code_build_encoder on host-only codes: k = n - rank(H) as an
    independent GF(2) basis computation gives it, for a lifted (4, 8) code
    (rank-deficient: each block row of an all-ones protograph lift sums to the
    same word) and an IRA code (full rank, k = n - m); bad sizes refused."""
    code, ent = I.qc_stand_in_code(256)
    h = ldpc.ldpc_code_create_qc(4, 8, 32, ent, device=-1)
    info, rank = gf2_information_positions(code.m, code.n, code.rows, code.cols)
    assert rank < code.m
    assert ldpc.ldpc_code_build_encoder(h) == code.n - rank == len(info)
    ira = I.mixed_codes()[0]
    hi = ldpc.ldpc_code_create(ira.m, ira.n, ira.rows, ira.cols, device=-1)
    info_i, rank_i = gf2_information_positions(ira.m, ira.n, ira.rows, ira.cols)
    assert rank_i == ira.m and info_i == list(range(ira.k))
    assert ldpc.ldpc_code_build_encoder(hi) == ira.k
    big = I.large_code_n64800()
    hb = ldpc.ldpc_code_create(big.m, big.n, big.rows, big.cols, device=-1)
    with pytest.raises(ldpc.LdpcError) as e:
        ldpc.ldpc_code_build_encoder(hb)
    assert e.value.status == -1 and "2^26" in str(e.value)
