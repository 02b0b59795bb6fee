"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module builds parity-check matrices, information words and codewords.
It holds none of the decoder's arithmetic and none of the channel-LLR
generator (each side implements that on its own); both the tests of the
CUDA path and the oracle tests draw their inputs from here.

Codes are irregular repeat-accumulate (IRA) LDPC codes, H = [H1 | H2]:

* H2 is the (m x m) dual-diagonal staircase (H2[i, i] = H2[i, i-1] = 1), so a
  codeword c = [u | p] is found by back-substitution p_i = s_i xor p_{i-1},
  s = H1 u (mod 2).
* H1 (m x k) is built by a seeded socket permutation: every information bit j
  owns deg_j variable sockets, every check i owns a near-equal share of the
  check sockets, the two socket lists are paired by a random permutation, and
  any repeated (check, bit) pair is repaired by random swaps so that H has no
  entry above 1.

The paper defines a code by its parity-check matrix H and its Tanner graph
(Section II-B, Eqs. 1-2); edges are the ones of H. The (14,7) example code of
Tables 1-2 is rebuilt from those tables in :func:`code_14_7`.
"""
from __future__ import annotations

import collections
import dataclasses
import math

import numpy as np
import scipy.sparse


@dataclasses.dataclass(frozen=True)
class Code:
    """A sparse parity-check matrix in COO form.

    ``rows[e], cols[e]`` is one nonzero of H. The COO order matters: the
    library and the oracle number edges by a stable sort of this list by
    column (edge ids of Table 1), so generated codes are emitted already
    sorted by (column, row).
    """

    m: int
    n: int
    rows: np.ndarray  # int32 [E]
    cols: np.ndarray  # int32 [E]
    name: str = ""
    k: int = -1  # information length of the systematic IRA layout (-1: unknown)

    @property
    def n_edges(self) -> int:
        return int(self.rows.shape[0])

    @property
    def rate(self) -> float:
        k = self.k if self.k >= 0 else self.n - self.m
        return k / self.n

    def dense(self) -> np.ndarray:
        """Dense uint8 H (small codes only)."""
        h = np.zeros((self.m, self.n), dtype=np.uint8)
        h[self.rows, self.cols] = 1
        return h


def largest_remainder(total: int, fractions: dict[int, float]) -> dict[int, int]:
    """Split ``total`` nodes over degrees by node-perspective fractions.

    Floors first, then the leftover nodes go to the largest remainders
    (ties broken towards the larger degree).
    """
    fsum = sum(fractions.values())
    exact = {d: total * f / fsum for d, f in fractions.items()}
    counts = {d: int(math.floor(x)) for d, x in exact.items()}
    left = total - sum(counts.values())
    order = sorted(exact, key=lambda d: (exact[d] - counts[d], d), reverse=True)
    for d in order[:left]:
        counts[d] += 1
    return counts


def _repair_duplicates(chk: np.ndarray, var: np.ndarray, rng: np.random.Generator, k: int) -> None:
    """Swap variable sockets until no (check, variable) pair repeats (in place)."""
    e1 = chk.shape[0]
    key = chk.astype(np.int64) * k + var
    uniq, inverse, counts = np.unique(key, return_inverse=True, return_counts=True)
    if np.all(counts == 1):
        return
    count = collections.Counter(key.tolist())
    dups = []
    seen_once = set()
    for idx in np.flatnonzero(counts[inverse] > 1).tolist():
        kk = int(key[idx])
        if kk in seen_once:
            dups.append(idx)
        else:
            seen_once.add(kk)
    for a in dups:
        for _try in range(100000):
            b = int(rng.integers(0, e1))
            if b == a:
                continue
            new_a = int(chk[a]) * k + int(var[b])
            new_b = int(chk[b]) * k + int(var[a])
            if count[new_a] or count[new_b] or new_a == new_b:
                continue
            count[int(chk[a]) * k + int(var[a])] -= 1
            count[int(chk[b]) * k + int(var[b])] -= 1
            var[a], var[b] = var[b], var[a]
            count[new_a] += 1
            count[new_b] += 1
            break
        else:  # pragma: no cover - astronomically unlikely for sparse codes
            raise RuntimeError("socket repair failed")


def ira_code(
    n: int,
    k: int,
    info_degrees: dict[int, float],
    seed: int,
    *,
    var_degree_overrides: dict[int, int] | None = None,
    check_h1_overrides: dict[int, int] | None = None,
    shuffle_degrees: bool = False,
    name: str = "",
) -> Code:
    """Seeded IRA code H = [H1 | H2] with a dual-diagonal staircase H2.

    ``info_degrees`` maps variable degree -> node fraction over the k
    information bits (rounded by largest remainder). ``var_degree_overrides``
    forces single information bits to a degree; ``check_h1_overrides`` forces
    the number of H1 sockets of single checks (its H2 part adds 2, or 1 for
    check 0). Remaining H1 sockets are spread as evenly as possible over the
    other checks, the extra ones on a seeded random subset.
    """
    m = n - k
    if m <= 0 or k <= 0:
        raise ValueError("need 0 < k < n")
    rng = np.random.default_rng(seed)
    counts = largest_remainder(k, info_degrees)
    degs = np.concatenate([np.full(c, d, dtype=np.int64) for d, c in sorted(counts.items(), reverse=True)])
    if shuffle_degrees:
        rng.shuffle(degs)
    for j, d in (var_degree_overrides or {}).items():
        degs[j] = d
    if np.any(degs > m):
        raise ValueError("variable degree exceeds the number of checks")
    e1 = int(degs.sum())
    var_sockets = np.repeat(np.arange(k, dtype=np.int64), degs)

    cdeg = np.zeros(m, dtype=np.int64)
    fixed = dict(check_h1_overrides or {})
    for i, d in fixed.items():
        cdeg[i] = d
    free = np.array([i for i in range(m) if i not in fixed], dtype=np.int64)
    rest = e1 - int(cdeg.sum())
    if rest < 0 or free.size == 0 and rest > 0:
        raise ValueError("check overrides exceed the H1 sockets")
    if free.size:
        base, extra = divmod(rest, free.size)
        cdeg[free] = base
        if extra:
            cdeg[rng.choice(free, size=extra, replace=False)] += 1
    chk_sockets = np.repeat(np.arange(m, dtype=np.int64), cdeg)
    var_perm = var_sockets[rng.permutation(e1)]
    _repair_duplicates(chk_sockets, var_perm, rng, k)

    rows = [chk_sockets, np.arange(m, dtype=np.int64), np.arange(1, m, dtype=np.int64)]
    cols = [var_perm, k + np.arange(m, dtype=np.int64), k + np.arange(m - 1, dtype=np.int64)]
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    order = np.lexsort((rows, cols))
    return Code(m=m, n=n, rows=rows[order].astype(np.int32), cols=cols[order].astype(np.int32),
                name=name or f"ira_n{n}_k{k}_s{seed}", k=k)


def encode_ira(code: Code, info: np.ndarray) -> np.ndarray:
    """Systematic IRA encoding, c = [u | p] with p the running XOR of H1 u.

    ``info`` is uint8 [F, k]; returns uint8 [F, n]. Only valid for codes made
    by :func:`ira_code` (H2 is the staircase in columns k..n-1).
    """
    k = code.k
    m = code.m
    info = np.asarray(info, dtype=np.uint8)
    sel = code.cols < k
    r1 = code.rows[sel].astype(np.int64)
    c1 = code.cols[sel].astype(np.int64)
    h1 = scipy.sparse.csr_matrix((np.ones(r1.shape[0], dtype=np.int64), (r1, c1)), shape=(m, k))
    s = np.asarray((h1 @ info.T.astype(np.int64)).T) & 1
    p = np.cumsum(s, axis=1) & 1
    return np.concatenate([info, p.astype(np.uint8)], axis=1)


def random_info(n_frames: int, k: int, seed: int) -> np.ndarray:
    """Bernoulli(1/2) information words, uint8 [n_frames, k]."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(n_frames, k), dtype=np.uint8)


def sigma2_from_ebn0(ebn0_db: float, rate: float) -> float:
    """Noise variance of unit-energy BPSK at Eb/N0 (dB): sigma^2 = (1/R) N0/2.

    With Es = 1 and Eb = Es / R, N0 = Eb / (Eb/N0), which gives the paper's
    sigma^2 = (1/R)(N0/2) of the BER-simulator section with Eb = 1/R folded in:
    sigma^2 = 1 / (2 R 10^(EbN0/10)).
    """
    return 1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))


def gaussian_llr(codewords: np.ndarray, sigma2: float, seed: int) -> np.ndarray:
    """CPU-side seeded BPSK/AWGN channel output for parity tests, float32 [F, n].

    x = 2c - 1 (bit 1 -> +1), y = x + sigma z, llr = 2 y / sigma^2, so that a
    positive LLR favours bit 1. Noise comes from numpy's PCG64, not from the
    on-device Philox generator, so decoder parity inputs never come from the
    CUDA path.
    """
    rng = np.random.default_rng(seed)
    cw = np.asarray(codewords, dtype=np.float64)
    y = (2.0 * cw - 1.0) + math.sqrt(sigma2) * rng.standard_normal(cw.shape)
    return (2.0 * y / sigma2).astype(np.float32)


# --- the paper's worked example -------------------------------------------------

# Table 1 (Section III-B), rows v and c: edge e joins variable V_14_7[e] and
# check C_14_7[e] of the (14,7) example code. The parity-check matrix itself is
# printed only as a figure; these two rows of the table define it.
V_14_7 = (0, 0, 0, 0, 1, 1, 2, 2, 3, 3, 3, 4, 4, 5, 5, 6, 6, 7, 7, 8, 8, 9, 9, 10, 10, 11, 11, 12, 12, 13, 13)
C_14_7 = (5, 3, 2, 0, 4, 0, 5, 1, 6, 4, 1, 4, 3, 1, 0, 4, 2, 6, 5, 5, 4, 2, 1, 6, 0, 3, 1, 6, 3, 5, 0)


def code_14_7() -> Code:
    """The (14,7) code of the paper's example, COO in Table 1's edge order.

    H has a one at (C_14_7[e], V_14_7[e]) for every edge e of Table 1. The
    COO keeps the table's order, so the edge ids the library assigns must
    reproduce e = 0..30.
    """
    return Code(m=7, n=14, rows=np.array(C_14_7, dtype=np.int32), cols=np.array(V_14_7, dtype=np.int32),
                name="paper_14_7", k=7)


# --- workloads ----------------------------------------------------------------------

def small_code_n1008(seed: int = 1008) -> Code:
    """n = 1008, rate 1/2, info degrees {2: 0.3, 3: 0.5, 8: 0.2}."""
    return ira_code(1008, 504, {2: 0.3, 3: 0.5, 8: 0.2}, seed, name="ira_n1008_r1/2")


def large_code_n64800(seed: int = 64800) -> Code:
    """n = 64800, rate 1/2, info degrees {8: 0.2, 3: 0.8}."""
    return ira_code(64800, 32400, {8: 0.2, 3: 0.8}, seed, name="ira_n64800_r1/2")


def tree_code(n_target: int, seed: int, max_check_degree: int = 4) -> Code:
    """Random code whose Tanner graph is a tree (cycle-free).

    Starting from variable 0, every new check joins one existing variable and
    1..max_check_degree-1 new variables, until n_target variables exist.
    """
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    n = 1
    m = 0
    while n < n_target:
        anchor = int(rng.integers(0, n))
        new = int(rng.integers(1, max_check_degree))
        new = min(new, n_target - n)
        members = [anchor] + list(range(n, n + new))
        for v in members:
            rows.append(m)
            cols.append(v)
        n += new
        m += 1
    rows = np.array(rows, dtype=np.int64)
    cols = np.array(cols, dtype=np.int64)
    order = np.lexsort((rows, cols))
    return Code(m=m, n=n, rows=rows[order].astype(np.int32), cols=cols[order].astype(np.int32),
                name=f"tree_n{n}_s{seed}", k=n - m)


def coo_code(m: int, n: int, rows, cols, name: str = "") -> Code:
    """A code from explicit COO lists (kept in the given order)."""
    return Code(m=m, n=n, rows=np.asarray(rows, dtype=np.int32), cols=np.asarray(cols, dtype=np.int32), name=name)


# --- quasi-cyclic (protograph-lifted) codes -----------------------------------------

def qc_code(mb: int, nb: int, Z: int, entries, name: str = "") -> Code:
    """Lift a base matrix with circulants: each (row, col, shift) entry puts
    P^shift at that block, row t joining column (t + shift) mod Z. COO order:
    entry-major, t-minor (the order the library's lifting entry uses)."""
    e = np.asarray(entries, dtype=np.int64).reshape(-1, 3)
    t = np.arange(Z, dtype=np.int64)
    rows = (e[:, 0:1] * Z + t[None, :]).reshape(-1)
    cols = (e[:, 1:2] * Z + (t[None, :] + e[:, 2:3]) % Z).reshape(-1)
    return Code(m=mb * Z, n=nb * Z, rows=rows.astype(np.int32), cols=cols.astype(np.int32),
                name=name or f"qc_{mb}x{nb}_Z{Z}")


def qc_regular_entries(dv: int, dc: int, Z: int, seed: int) -> list[tuple[int, int, int]]:
    """All-ones dv x dc base matrix with seeded circulant shifts: a (dv, dc)-
    regular QC code of design rate 1 - dv/dc and dv * Z * dc edges."""
    rng = np.random.default_rng(seed)
    return [(i, j, int(rng.integers(0, Z))) for i in range(dv) for j in range(dc)]


def qc_stand_in_code(n: int, seed: int | None = None) -> tuple[Code, list]:
    """Rate-1/2 (4, 8)-regular QC stand-in of length n (4 edges per bit), the
    protograph-lifted counterpart of the paper's benchmark family."""
    if n % 8:
        raise ValueError("n must be a multiple of 8")
    Z = n // 8
    ent = qc_regular_entries(4, 8, Z, seed if seed is not None else n + 1)
    return qc_code(4, 8, Z, ent, name=f"qc48_n{n}_Z{Z}"), ent


# --- mixed-code workload: 8 codes of different lengths, rates and degrees --------

MIXED_SPECS = (  # (n, k, name); the 8192-bit code carries a degree-64 variable and a degree-96 check
    (576, 480, "n576_r5/6"),
    (1152, 864, "n1152_r3/4"),
    (2304, 1536, "n2304_r2/3"),
    (4096, 2048, "n4096_r1/2"),
    (8192, 6144, "n8192_r3/4_deg64_96"),
    (16200, 5400, "n16200_r1/3"),
    (32400, 21600, "n32400_r2/3"),
    (64800, 54000, "n64800_r5/6"),
)


def mixed_codes() -> list[Code]:
    """The eight seeded IRA codes of the mixed-code workload, shortest first.

    Info-bit degrees {3: 0.8, 4: 0.2}; check degrees follow from the rate
    (about 3-4 at rate 1/3 up to about 18 at rate 5/6). Code 4 (n = 8192) has
    one information bit of degree 64 and one check of degree 96 (94 H1
    sockets plus its two staircase ones).
    """
    return [mixed_code(idx) for idx in range(len(MIXED_SPECS))]


def mixed_code(idx: int) -> Code:
    """Code ``idx`` of :func:`mixed_codes` alone (seed 100 + idx)."""
    n, k, name = MIXED_SPECS[idx]
    over_v = {0: 64} if n == 8192 else None
    over_c = {5: 94} if n == 8192 else None
    return ira_code(n, k, {3: 0.8, 4: 0.2}, seed=100 + idx, var_degree_overrides=over_v,
                    check_h1_overrides=over_c, name=name)


def zipf_frames(total: int, count: int, s: float = 1.1) -> list[int]:
    """Split `total` frames over `count` ranks with Zipf(s) weights (rank 1
    gets the most), by largest remainder."""
    weights = {r: r ** (-s) for r in range(1, count + 1)}
    split = largest_remainder(total, weights)
    return [split[r] for r in range(1, count + 1)]
