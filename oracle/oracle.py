"""Python face of the FP64 CPU oracle (test infrastructure).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module. The product path (the
CUDA library and its binding) never imports or calls it, and this module
never imports the product package's compute code.

Contents, each following the paper (arXiv:1609.01567):

* :func:`decode`, :func:`sp_pass`, :func:`syndrome_weight`,
  :func:`address_iterators`, :func:`gen_awgn`, :func:`philox_blocks` --
  ctypes wrappers over ``ldpc_oracle.c`` (Algorithms 1-6 in the LLR domain,
  Tables 1-2, the BER-simulator channel of Section IV).
* :func:`decode_probability_domain` -- a second, literal oracle that runs
  Algorithms 1, 3, 4 and 6 on probabilities (normalised), used only to pin the
  LLR rewrite where nothing saturates.
* :func:`codewords_of`, :func:`map_llr`, :func:`ml_decode` -- brute force over
  all codewords of tiny codes (exact bitwise MAP marginals and ML decoding).
"""
from __future__ import annotations

import ctypes
import itertools
import os
from pathlib import Path

import numpy as np

from . import build as _build

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.library_path()
        if not path.exists():
            _build.build()
        lib = ctypes.CDLL(str(path))
        i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        vp = ctypes.c_void_p
        lib.orc_decode.argtypes = [i32, i32, i64, vp, vp, vp, i32, i32, i32, dbl, vp, vp, vp, vp, vp, i32, i32, dbl, dbl,
                                   i32, dbl, i32, vp, vp, i32]
        lib.orc_decode.restype = ctypes.c_int
        lib.orc_pass.argtypes = [i32, i32, i64, vp, vp, vp, i32, vp, dbl, vp, vp, vp, vp, i32, i32, dbl, dbl, i32, dbl,
                                 i32, vp, vp, i32]
        lib.orc_store.argtypes = [dbl, i32, dbl, i32]
        lib.orc_store.restype = dbl
        lib.orc_pass.restype = ctypes.c_int
        lib.orc_phi.argtypes = [dbl]
        lib.orc_phi.restype = dbl
        lib.orc_phi_chord.argtypes = [dbl]
        lib.orc_phi_chord.restype = dbl
        lib.orc_syndrome.argtypes = [i32, i32, i64, vp, vp, vp, i32, vp]
        lib.orc_syndrome.restype = ctypes.c_int
        lib.orc_address_iterators.argtypes = [i32, i32, i64, vp, vp] + [vp] * 11
        lib.orc_address_iterators.restype = ctypes.c_int
        lib.orc_philox_blocks.argtypes = [u64, u64, u64, u64, i64, vp]
        lib.orc_philox_blocks.restype = None
        lib.orc_gen_awgn.argtypes = [u64, i64, i32, i32, dbl, vp, vp]
        lib.orc_gen_awgn.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _coo(code):
    rows = np.ascontiguousarray(code.rows, dtype=np.int32)
    cols = np.ascontiguousarray(code.cols, dtype=np.int32)
    return rows, cols


def default_threads() -> int:
    return int(os.environ.get("LDPC_ORACLE_THREADS", "1"))


RULES = {"sp": 0, "min_sum": 1, "sp_table": 2, "min_sum_adaptive": 3}

# Stored-message formats: (format, lattice step, largest |level|). "f64"
# keeps the messages unrounded, "i8" stores k * 20/127 with |k| <= 127,
# "f16" and "bf16" round to IEEE binary16 and bfloat16 (nearest, ties to even).
MSG = {"f64": (0, 0.0, 0), "i8": (1, 20.0 / 127.0, 127), "f16": (2, 0.0, 0), "bf16": (3, 0.0, 0)}


def _msg(msg):
    if isinstance(msg, tuple):  # a lattice (step, levels)
        return 1, float(msg[0]), int(msg[1])
    return MSG[msg]


def store(r: float, msg) -> float:
    """The stored value of one message under storage format ``msg``."""
    return _lib().orc_store(float(r), *_msg(msg))


def _degree_tables(rule, alpha_by_degree, beta_by_degree):
    """The per-check-degree scale and offset of rule "min_sum_adaptive"
    (index = check degree; degrees past the end take the last entry), as
    FP64 arrays kept alive by the caller, plus their length."""
    if rule != "min_sum_adaptive":
        return None, None, 0
    a = np.ascontiguousarray(alpha_by_degree, dtype=np.float64)
    b = np.ascontiguousarray(beta_by_degree if beta_by_degree is not None else np.zeros_like(a), dtype=np.float64)
    if a.ndim != 1 or a.shape != b.shape:
        raise ValueError("alpha_by_degree and beta_by_degree must be 1-D and of one length")
    return a, b, int(a.shape[0])


def decode(code, llr, max_iter: int, *, early_exit: bool = True, l_max: float = 20.0,
           want_post: bool = True, want_r: bool = False, n_threads: int | None = None,
           rule: str = "sp", alpha: float = 1.0, beta: float = 0.0, msg="f64", alpha_by_degree=None,
           beta_by_degree=None):
    """Sum-product decode (Algorithm 2) of LLRs ``llr`` [F, n] in FP64
    (``rule="min_sum"``: the min-sum family, |r| = clamp(alpha min - beta);
    ``rule="min_sum_adaptive"``: the same with alpha and beta taken per check
    degree d from ``alpha_by_degree[min(d, len - 1)]`` and ``beta_by_degree``;
    ``rule="sp_table"``: sum-product with phi on the chords of a log-spaced
    grid, 64 buckets per octave;
    ``msg``: a key of :data:`MSG` or a (step, levels) pair for quantised
    message storage).

    Returns a dict with ``bits`` uint8 [F, n], ``iters`` int32 [F], ``ok``
    uint8 [F], and optionally ``post`` float64 [F, n] (APP LLRs) and ``r``
    float64 [F, E] (last check-to-bit messages in edge order).
    """
    lam = np.ascontiguousarray(llr, dtype=np.float64)
    f, n = lam.shape
    assert n == code.n
    rows, cols = _coo(code)
    e = rows.shape[0]
    bits = np.zeros((f, n), dtype=np.uint8)
    iters = np.zeros(f, dtype=np.int32)
    ok = np.zeros(f, dtype=np.uint8)
    post = np.zeros((f, n), dtype=np.float64) if want_post else None
    r = np.zeros((f, e), dtype=np.float64) if want_r else None
    ad, bd, nd = _degree_tables(rule, alpha_by_degree, beta_by_degree)
    rc = _lib().orc_decode(code.m, code.n, e, _ptr(rows), _ptr(cols), _ptr(lam), f, max_iter,
                           1 if early_exit else 0, l_max, _ptr(bits), _ptr(iters), _ptr(ok), _ptr(post),
                           _ptr(r), n_threads if n_threads is not None else default_threads(), RULES[rule],
                           alpha, beta, *_msg(msg), _ptr(ad), _ptr(bd), nd)
    if rc != 0:
        raise ValueError("oracle decode rejected its input")
    out = {"bits": bits, "iters": iters, "ok": ok}
    if want_post:
        out["post"] = post
    if want_r:
        out["r"] = r
    return out


def sp_pass(code, llr, r_prev=None, *, l_max: float = 20.0, n_threads: int | None = None, rule: str = "sp",
            alpha: float = 1.0, beta: float = 0.0, msg="f64", alpha_by_degree=None, beta_by_degree=None):
    """One flooding pass from messages ``r_prev`` [F, E] (None: first pass).

    Returns ``r`` [F, E], ``post`` [F, n], ``bits`` [F, n], ``weight`` [F].
    """
    lam = np.ascontiguousarray(llr, dtype=np.float64)
    f, n = lam.shape
    rows, cols = _coo(code)
    e = rows.shape[0]
    rp = None if r_prev is None else np.ascontiguousarray(r_prev, dtype=np.float64)
    r = np.zeros((f, e), dtype=np.float64)
    app = np.zeros((f, n), dtype=np.float64)
    bits = np.zeros((f, n), dtype=np.uint8)
    w = np.zeros(f, dtype=np.int64)
    ad, bd, nd = _degree_tables(rule, alpha_by_degree, beta_by_degree)
    rc = _lib().orc_pass(code.m, code.n, e, _ptr(rows), _ptr(cols), _ptr(lam), f, _ptr(rp), l_max, _ptr(r),
                         _ptr(app), _ptr(bits), _ptr(w), n_threads if n_threads is not None else default_threads(),
                         RULES[rule], alpha, beta, *_msg(msg), _ptr(ad), _ptr(bd), nd)
    if rc != 0:
        raise ValueError("oracle pass rejected its input")
    return {"r": r, "post": app, "bits": bits, "weight": w}


def phi(x: float) -> float:
    """phi(x) = ln((e^x + 1)/(e^x - 1)) as the oracle evaluates it."""
    return _lib().orc_phi(float(x))


def phi_chord(x: float) -> float:
    """The tabulated phi of rule "sp_table" (chords on 64 buckets per octave)."""
    return _lib().orc_phi_chord(float(x))


def syndrome_weight(code, bits) -> np.ndarray:
    """Number of unsatisfied checks of each hard word ``bits`` [F, n]."""
    b = np.ascontiguousarray(bits, dtype=np.uint8)
    if b.ndim == 1:
        b = b[None]
    rows, cols = _coo(code)
    w = np.zeros(b.shape[0], dtype=np.int64)
    rc = _lib().orc_syndrome(code.m, code.n, rows.shape[0], _ptr(rows), _ptr(cols), _ptr(b), b.shape[0], _ptr(w))
    if rc != 0:
        raise ValueError("oracle syndrome rejected its input")
    return w


ITERATOR_NAMES = ("v", "c", "t", "s", "u", "ebar", "vbar", "cbar", "tbar", "sbar", "ubar")


def address_iterators(code) -> dict[str, np.ndarray]:
    """The paper's address-iterator arrays (Tables 1-2) of ``code``."""
    rows, cols = _coo(code)
    e = rows.shape[0]
    arrs = {k: np.zeros(e, dtype=np.int32) for k in ITERATOR_NAMES}
    rc = _lib().orc_address_iterators(code.m, code.n, e, _ptr(rows), _ptr(cols),
                                      *[_ptr(arrs[k]) for k in ITERATOR_NAMES])
    if rc != 0:
        raise ValueError("bad code")
    arrs["e"] = np.arange(e, dtype=np.int32)
    return arrs


def philox_blocks(key0: int, key1: int, ctr0: int, ctr1: int, count: int) -> np.ndarray:
    """Philox-4x64-10 blocks for counters (ctr0 + i, ctr1, 0, 0): uint64 [count, 4]."""
    out = np.zeros((count, 4), dtype=np.uint64)
    _lib().orc_philox_blocks(key0, key1, ctr0, ctr1, count, _ptr(out))
    return out


def gen_awgn(seed: int, frame_offset: int, n_frames: int, n: int, sigma2: float, codewords=None) -> np.ndarray:
    """BPSK/AWGN channel LLRs [F, n] in FP64 (Philox-4x64-10 + Box-Muller)."""
    cw = None if codewords is None else np.ascontiguousarray(codewords, dtype=np.uint8)
    if cw is not None:
        assert cw.shape == (n_frames, n)
    out = np.zeros((n_frames, n), dtype=np.float64)
    rc = _lib().orc_gen_awgn(seed, frame_offset, n_frames, n, sigma2, _ptr(cw), _ptr(out))
    if rc != 0:
        raise ValueError("bad generator arguments")
    return out


# ----------------------------------------------------------------------------------
# Literal probability-domain oracle (Algorithms 1, 3, 4, 6 with normalised q)
# ----------------------------------------------------------------------------------

def decode_probability_domain(code, y, sigma2: float, n_passes: int):
    """Run Algorithm 2's passes on probabilities, without early exit.

    Algorithm 3: p_j = 1 / (1 + exp(-2 y_j / sigma^2)) = P(c_j = 1), q_ij = p_j.
    Algorithm 1, second half: r0_ij = 1/2 + 1/2 prod_{j' != j} (1 - 2 q1_ij'),
    r1_ij = 1 - r0_ij. First half: q_ij proportional to
    p_j prod_{i' != i} r_i'j (for both values of the bit), normalised so that
    q0 + q1 = 1. Algorithm 4: Q_j = p_j prod_i r_ij, bit 1 iff Q1 > Q0 -- the
    tie is sent to 0 here as in Algorithm 5 -- and Algorithm 6 xors the bits of
    every check.

    Returns the list, one entry per pass, of (r1 [F, E], Q1 [F, n] normalised,
    bits [F, n], syndrome weight [F]). Edge order is the oracle's (Table 1).
    """
    y = np.asarray(y, dtype=np.float64)
    f, n = y.shape
    it = address_iterators(code)
    v, c, ebar, cbar = it["v"], it["c"], it["ebar"], it["cbar"]
    e_count = v.shape[0]
    p1 = 1.0 / (1.0 + np.exp(-2.0 * y / sigma2))
    p0 = 1.0 - p1
    q1 = p1[:, v].copy()
    out = []
    r0 = r1 = None
    for step in range(n_passes + 1):
        if step > 0:
            # Values to Check Nodes (first half of an iteration)
            a1 = np.empty((f, e_count))
            a0 = np.empty((f, e_count))
            for e in range(e_count):
                j = v[e]
                others = [e2 for e2 in np.flatnonzero(v == j) if e2 != e]
                a1[:, e] = p1[:, j] * np.prod(r1[:, others], axis=1)
                a0[:, e] = p0[:, j] * np.prod(r0[:, others], axis=1)
            q1 = a1 / (a0 + a1)
        # Values to Variable Nodes (second half of an iteration)
        r0 = np.empty((f, e_count))
        for k in range(e_count):
            e = ebar[k]
            i = cbar[k]
            others = [ebar[k2] for k2 in np.flatnonzero(cbar == i) if ebar[k2] != e]
            r0[:, e] = 0.5 + 0.5 * np.prod(1.0 - 2.0 * q1[:, others], axis=1)
        r1 = 1.0 - r0
        # Calculate Estimation
        big_q1 = p1.copy()
        big_q0 = p0.copy()
        for e in range(e_count):
            big_q1[:, v[e]] *= r1[:, e]
            big_q0[:, v[e]] *= r0[:, e]
        bits = (big_q1 > big_q0).astype(np.uint8)
        # Calculate Syndrome
        z = np.zeros((f, code.m), dtype=np.uint8)
        for e in range(e_count):
            z[:, c[e]] ^= bits[:, v[e]]
        out.append((r1.copy(), big_q1 / (big_q0 + big_q1), bits, z.sum(axis=1)))
    return out


# ----------------------------------------------------------------------------------
# Brute force over all codewords (n <= ~20)
# ----------------------------------------------------------------------------------

def codewords_of(code) -> np.ndarray:
    """All codewords of H (uint8 [2^k, n]) by Gaussian elimination over GF(2)."""
    h = code.dense().astype(np.uint8) % 2
    m, n = h.shape
    a = h.copy()
    pivots = []
    row = 0
    for col in range(n):
        piv = None
        for r in range(row, m):
            if a[r, col]:
                piv = r
                break
        if piv is None:
            continue
        a[[row, piv]] = a[[piv, row]]
        for r in range(m):
            if r != row and a[r, col]:
                a[r] ^= a[row]
        pivots.append(col)
        row += 1
        if row == m:
            break
    free = [c for c in range(n) if c not in pivots]
    basis = []
    for fc in free:
        vec = np.zeros(n, dtype=np.uint8)
        vec[fc] = 1
        for r, pc in enumerate(pivots):
            vec[pc] = a[r, fc]
        basis.append(vec)
    basis = np.array(basis, dtype=np.uint8).reshape(len(free), n)
    words = []
    for coeffs in itertools.product((0, 1), repeat=len(free)):
        cw = np.zeros(n, dtype=np.uint8)
        for cf, b in zip(coeffs, basis):
            if cf:
                cw ^= b
        words.append(cw)
    return np.array(words, dtype=np.uint8)


def map_llr(codewords: np.ndarray, llr: np.ndarray) -> np.ndarray:
    """Exact bitwise MAP LLRs ln(sum_{c: c_j=1} P(c|y) / sum_{c: c_j=0} P(c|y)).

    With lambda = ln(P1/P0) per bit and a uniform prior over codewords,
    P(c | y) is proportional to exp(sum_j c_j lambda_j).
    """
    lam = np.atleast_2d(np.asarray(llr, dtype=np.float64))
    cw = codewords.astype(np.float64)
    score = lam @ cw.T  # [F, W]
    smax = score.max(axis=1, keepdims=True)
    wts = np.exp(score - smax)
    num = wts @ cw
    den = wts @ (1.0 - cw)
    return np.log(num) - np.log(den)


def ml_decode(codewords: np.ndarray, llr: np.ndarray) -> np.ndarray:
    """ML codeword per frame: argmax over codewords of sum_j c_j lambda_j."""
    lam = np.atleast_2d(np.asarray(llr, dtype=np.float64))
    score = lam @ codewords.astype(np.float64).T
    return codewords[np.argmax(score, axis=1)]


def library_path() -> Path:
    return _build.library_path()
