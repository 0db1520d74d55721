"""Pins for the CPU oracle, checked against what the paper and mathematics fix.

Nothing here re-types the oracle's formulas: values come from the paper's
worked examples (tests/golden/, each citing its passage), from closed forms
(identity, permutation, empty, dense products of small integers, exact
rational sums), from invariants, or from a brute-force re-derivation of the
index artefacts through a per-entry row-id expansion (a different computation
from the oracle's merge and row-pointer scans).
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from conftest import GOLDEN

U = 2.0 ** -53  # unit roundoff of FP64


def gamma(n):
    return n * U / (1 - n * U)


# ---------------------------------------------------------------------------
# the 6x6 example of Sec. 2.1

def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_example_6x6_product_closed_form():
    g = _load("paper_example_6x6.json")
    # substitute distinct small integers for the symbols a..l: every product
    # and sum is then exact in FP64, so equality is bit-exact
    sub = {s: float(3 + 2 * i) for i, s in enumerate(g["val_symbols"])}
    val = np.array([sub[s] for s in g["val_symbols"]])
    y = oracle.spmv(g["row_ptr"], g["col_idx"], val, np.array(g["x"], dtype=float))
    want = [sum(c * sub[s] for s, c in coeffs.items()) for coeffs in g["y_coefficients"]]
    assert y.tolist() == want
    y_omp, _ = oracle.spmv_omp(g["row_ptr"], g["col_idx"], val, np.array(g["x"], dtype=float))
    assert y_omp.tolist() == want
    y2, s = oracle.spmv_dot2(g["row_ptr"], g["col_idx"], val, np.array(g["x"], dtype=float))
    assert y2.tolist() == want


def test_example_6x6_descriptor_and_dirty():
    g = _load("paper_example_6x6.json")
    # one tile covering all 12 entries (any W*T >= 12)
    for L in (12, 16, 32):
        d = oracle.descriptors(g["row_ptr"], L)
        assert d.shape[0] == 1
        bits = [(int(d[0, k // 32]) >> (k % 32)) & 1 for k in range(12)]
        assert bits == g["segment_descriptor"]
        # nothing set past the last entry
        assert all(((int(d[0, k // 32]) >> (k % 32)) & 1) == 0 for k in range(12, L))
        dirty, nseg = oracle.tile_flags(g["row_ptr"], L)
        assert dirty.tolist() == [1]          # row 3 is empty
        assert nseg.tolist() == [sum(g["segment_descriptor"])]


def test_example_6x6_two_stages_match_definition():
    g = _load("paper_example_6x6.json")
    sub = {s: float(2 + i) for i, s in enumerate(g["val_symbols"])}
    val = np.array([sub[s] for s in g["val_symbols"]])
    x = np.array(g["x"], dtype=float)
    want = oracle.spmv(g["row_ptr"], g["col_idx"], val, x)
    for T, W, S in [(1, 1, 1), (2, 1, 1), (2, 2, 1), (1, 3, 2), (4, 3, 1), (2, 2, 3), (1, 12, 1)]:
        st = oracle.speculative_stage(g["row_ptr"], g["col_idx"], val, x, T, W, S)
        y = oracle.checking_stage(g["row_ptr"], T, W, S, st)
        assert y.tolist() == want.tolist(), (T, W, S)


# ---------------------------------------------------------------------------
# the 12-row example of Sec. 3.2 (Fig. 2)

def _example12(split=(9, 14)):
    g = _load("paper_example_12row.json")
    rp = [None] * 13
    for k, v in g["row_ptr_printed"].items():
        rp[int(k)] = v
    rp[2], rp[3] = split        # not printed: rows 1..3 non-empty (only rows 6, 9 are)
    assert 3 < rp[2] < rp[3] < 19
    assert all(v is not None for v in rp)
    letters = g["row_letters"]
    letter_val = {c: float(i + 2) for i, c in enumerate("abcdefghij")}
    nnz = rp[-1]
    val = np.empty(nnz)
    col = np.zeros(nnz, dtype=np.int32)
    for r in range(12):
        for k in range(rp[r], rp[r + 1]):
            val[k] = letter_val[letters[r]]
            col[k] = k % 12                  # any column: x = 1 everywhere
    x = np.ones(12)
    return g, np.array(rp, dtype=np.int32), col, val, x, letter_val


def _sym(expr, letter_val):
    return float(int(expr[:-1])) * letter_val[expr[-1]]


@pytest.mark.parametrize("split", [(9, 14), (4, 5), (17, 18), (5, 12)])
def test_example12_tile_offsets_and_descriptor(split):
    g, rp, col, val, x, lv = _example12(split)
    L = g["T"] * g["W"]
    assert (rp[4:13] - g["boundaries"][1]).tolist() == g["tile2_row_ptr_minus_boundary"]
    assert oracle.tile_offsets(rp, L).tolist() == g["tile_offset"]
    d = oracle.descriptors(rp, L)
    heads = [k for k in range(L) if (int(d[1, k // 32]) >> (k % 32)) & 1]
    assert heads == g["tile2_effective_heads"]           # raw: bit 0 not forced
    assert sorted(set(heads) | {0}) == g["tile2_descriptor_final_heads"]
    dirty, nseg = oracle.tile_flags(rp, L)
    assert int(dirty.sum()) == g["dirty_counter"]
    toff = oracle.tile_offsets(rp, L)
    spec = [[int(toff[t]), int(toff[t + 1])] for t in np.nonzero(dirty)[0]]
    assert spec == g["speculator"]


@pytest.mark.parametrize("split", [(9, 14), (4, 5), (17, 18)])
def test_example12_speculative_stage(split):
    g, rp, col, val, x, lv = _example12(split)
    T, W, S = g["T"], g["W"], g["S"]
    st = oracle.speculative_stage(rp, col, val, x, T, W, S)
    assert st["dirty_counter"] == g["dirty_counter"]
    toff = oracle.tile_offsets(rp, T * W)
    assert [[int(toff[t]), int(toff[t + 1])] for t in st["speculator"]] == g["speculator"]
    # first partial 3a goes to the synchronizer with index 0
    assert int(st["sync_idx"][0]) == g["synchronizer_first"]["idx"]
    assert st["sync_val"][0] == _sym(g["synchronizer_first"]["value"], lv)
    # 5e is carried from tile 1 into tile 2, whose first segment (row 4) then
    # holds 5e + 3e
    assert st["y"][4] == _sym(g["transmitted_from_tile1"], lv) + 3 * lv["e"]
    # after synchronisation the four partials of rows 7, 8, 10, 11 sit in
    # slots 6..9
    y_sync = st["y"].copy()
    y_sync[st["sync_idx"]] += st["sync_val"]
    for slot, expr in g["misplaced_after_synchronization"].items():
        assert y_sync[int(slot)] == _sym(expr, lv)
    # checking stage puts them in their rows and zeroes the empty rows
    y = oracle.checking_stage(rp, T, W, S, st)
    for expr, row in g["rows_of_misplaced"].items():
        assert y[row] == _sym(expr, lv)
    assert y[6] == 0.0 and y[9] == 0.0
    assert y.tolist() == oracle.spmv(rp, col, val, x).tolist()


# ---------------------------------------------------------------------------
# brute force over every short row-length pattern: index artefacts derived a
# second way, from the row id of each entry

def _brute_artefacts(lengths, L):
    m = len(lengths)
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=rp[1:])
    nnz = int(rp[-1])
    rowid = np.repeat(np.arange(m), lengths)
    nt = (nnz + L - 1) // L
    b = [min(t * L, nnz) for t in range(nt + 1)]
    start = [int(rowid[bt]) if bt < nnz else m for bt in b]
    desc, dirty, nseg = [], [], []
    for t in range(nt):
        lo, hi = b[t], b[t + 1]
        bits = []
        for k in range(hi - lo):
            p = lo + k
            if k == 0:
                bits.append(int(rp[rowid[p]] == p))
            else:
                bits.append(int(rowid[p] != rowid[p - 1]))
        desc.append(bits)
        rows_in = set(rowid[lo:hi].tolist())
        nseg.append(len(rows_in))
        dirty.append(int(any(r not in rows_in for r in range(start[t], start[t + 1]))))
    return rp.astype(np.int32), start, desc, dirty, nseg


def _patterns():
    for m in range(0, 6):
        for lens in itertools.product(range(4), repeat=m):
            yield list(lens)


def test_bruteforce_index_artefacts():
    count = 0
    for lens in _patterns():
        for L in (1, 2, 3, 4, 5, 8):
            rp, start, desc, dirty, nseg = _brute_artefacts(lens, L)
            toff = oracle.tile_offsets(rp, L)
            assert toff.tolist() == start, (lens, L)
            nt = len(start) - 1
            if nt == 0:
                continue
            d = oracle.descriptors(rp, L)
            got = [[(int(d[t, k // 32]) >> (k % 32)) & 1 for k in range(len(desc[t]))]
                   for t in range(nt)]
            assert got == desc, (lens, L)
            # positions past the end of the last tile stay clear
            last = len(desc[-1])
            assert all(((int(d[nt - 1, k // 32]) >> (k % 32)) & 1) == 0 for k in range(last, L))
            df, ns = oracle.tile_flags(rp, L)
            assert df.tolist() == dirty, (lens, L)
            assert ns.tolist() == nseg, (lens, L)
            count += 1
    assert count > 5000


def test_bruteforce_two_stages_equal_definition():
    rng = np.random.Generator(np.random.PCG64(7))
    checked = 0
    for lens in _patterns():
        if len(lens) == 0 or sum(lens) == 0:
            continue
        if rng.random() > 0.35:
            continue
        nnz = sum(lens)
        rp = np.zeros(len(lens) + 1, dtype=np.int32)
        np.cumsum(lens, out=rp[1:])
        n = 4
        col = rng.integers(0, n, size=nnz).astype(np.int32)
        val = rng.integers(-4, 5, size=nnz).astype(float)
        x = rng.integers(-3, 4, size=n).astype(float)
        want = oracle.spmv(rp, col, val, x)
        for T, W, S in [(1, 1, 1), (2, 1, 2), (1, 2, 1), (2, 2, 2), (3, 1, 1), (1, 3, 3)]:
            st = oracle.speculative_stage(rp, col, val, x, T, W, S)
            y = oracle.checking_stage(rp, T, W, S, st)
            assert y.tolist() == want.tolist(), (lens, T, W, S)
            toff = oracle.tile_offsets(rp, T * W)
            dirty, _ = oracle.tile_flags(rp, T * W)
            assert sorted(st["speculator"].tolist()) == np.nonzero(dirty)[0].tolist()
            nb = oracle.bunch_count(nnz, T, W, S)
            assert st["sync_idx"].tolist() == [int(toff[w * S]) for w in range(nb)]
            checked += 1
    assert checked > 500


# ---------------------------------------------------------------------------
# closed forms and invariants of y = A x

def _dense(rp, col, val, m, n):
    D = np.zeros((m, n))
    for r in range(m):
        for k in range(rp[r], rp[r + 1]):
            D[r, col[k]] += val[k]
    return D


def test_dense_small_integers_exact():
    rng = np.random.Generator(np.random.PCG64(11))
    for trial in range(40):
        m, n = int(rng.integers(1, 30)), int(rng.integers(1, 30))
        lens = rng.integers(0, n + 3, size=m)          # duplicates allowed
        rp = np.zeros(m + 1, dtype=np.int32)
        np.cumsum(lens, out=rp[1:])
        nnz = int(rp[-1])
        col = rng.integers(0, n, size=nnz).astype(np.int32)
        val = rng.integers(-9, 10, size=nnz).astype(float)
        x = rng.integers(-9, 10, size=n).astype(float)
        D = _dense(rp, col, val, m, n)
        want = D @ x                                   # exact: small integers
        assert oracle.spmv(rp, col, val, x).tolist() == want.tolist()
        assert oracle.spmv_dot2(rp, col, val, x)[0].tolist() == want.tolist()


def test_identity_permutation_empty():
    n = 257
    x = synth.sym_vector(n, seed=5)
    rp = np.arange(n + 1, dtype=np.int32)
    eye = oracle.spmv(rp, np.arange(n, dtype=np.int32), np.ones(n), x)
    assert eye.tolist() == x.tolist()
    perm = np.random.Generator(np.random.PCG64(3)).permutation(n).astype(np.int32)
    assert oracle.spmv(rp, perm, np.ones(n), x).tolist() == x[perm].tolist()
    empty = np.zeros(n + 1, dtype=np.int32)
    y = oracle.spmv(empty, np.zeros(0, np.int32), np.zeros(0), x)
    assert y.tolist() == [0.0] * n and not np.signbit(y).any()
    y, s = oracle.spmv_dot2(empty, np.zeros(0, np.int32), np.zeros(0), x)
    assert y.tolist() == [0.0] * n and s.tolist() == [0.0] * n


def _exact_row_sums(rp, col, val, x, rows):
    out = []
    for r in rows:
        acc = Fraction(0)
        for k in range(rp[r], rp[r + 1]):
            acc += Fraction(val[k]) * Fraction(x[col[k]])
        out.append(acc)
    return out


def test_single_long_row_against_exact_rational():
    n = 5000
    rng = np.random.Generator(np.random.PCG64(21))
    col = np.sort(rng.choice(n, size=3000, replace=False)).astype(np.int32)
    val = rng.uniform(-1, 1, size=3000)
    x = rng.uniform(-1, 1, size=n)
    rp = np.array([0, 3000], dtype=np.int32)
    exact = _exact_row_sums(rp, col, val, x, [0])[0]
    y = oracle.spmv(rp, col, val, x)[0]
    yd, s = oracle.spmv_dot2(rp, col, val, x)
    absprod = float(sum(abs(Fraction(val[k]) * Fraction(x[col[k]])) for k in range(3000)))
    # plain loop: |y - exact| <= gamma_n * sum |a x|  (Higham, Accuracy and
    # Stability, eq. 3.5)
    assert abs(Fraction(y) - exact) <= Fraction(gamma(3000) * absprod)
    # Dot2: |res - exact| <= u |exact| + gamma_n^2 sum |a x|  (Ogita-Rump-Oishi,
    # Prop. 5.5 with K = 2)
    bound = U * abs(float(exact)) + gamma(3000) ** 2 * absprod
    assert abs(Fraction(yd[0]) - exact) <= Fraction(bound) * (1 + 1e-12)
    assert abs(s[0] - absprod) <= gamma(3000) * absprod


def test_dot2_rows_against_exact_rational():
    A = synth.from_lengths(synth.random_lengths(60, seed=4, mean=30, p_empty=0.2), 200, seed=4)
    x = synth.sym_vector(200, seed=9)
    yd, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
    y = oracle.spmv(A.row_ptr, A.col, A.val, x)
    ex = _exact_row_sums(A.row_ptr, A.col, A.val, x, range(A.m))
    for r in range(A.m):
        nr = int(A.row_ptr[r + 1] - A.row_ptr[r])
        if nr == 0:
            assert yd[r] == 0.0 and y[r] == 0.0 and s[r] == 0.0
            continue
        bound = U * abs(float(ex[r])) + gamma(nr) ** 2 * s[r] * 1.01
        assert abs(Fraction(yd[r]) - ex[r]) <= Fraction(bound)
        assert abs(Fraction(y[r]) - ex[r]) <= Fraction(gamma(nr) * s[r] * 1.01)


def test_column_sum_invariant():
    """1^T (A x) = (1^T A) x, checked in exact rationals on the oracle's y
    within the row loop's rounding bound."""
    A = synth.from_lengths(synth.random_lengths(300, seed=12, mean=12, p_empty=0.1), 150, seed=12)
    x = synth.sym_vector(150, seed=13)
    y = oracle.spmv(A.row_ptr, A.col, A.val, x)
    lhs = sum(Fraction(v) for v in y)
    colsum = [Fraction(0)] * A.n
    for k in range(A.nnz):
        colsum[A.col[k]] += Fraction(A.val[k])
    rhs = sum(colsum[j] * Fraction(x[j]) for j in range(A.n))
    _, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
    maxlen = int(np.diff(A.row_ptr).max())
    assert abs(lhs - rhs) <= Fraction(gamma(maxlen) * float(s.sum()) * 1.01)


def test_omp_equals_serial():
    A = synth.from_lengths(synth.random_lengths(5000, seed=2, mean=9, p_empty=0.3), 4000, seed=2)
    x = synth.sym_vector(4000, seed=3)
    y = oracle.spmv(A.row_ptr, A.col, A.val, x)
    for nt in (1, 2, 3):
        y2, used = oracle.spmv_omp(A.row_ptr, A.col, A.val, x, nthreads=nt)
        assert used == nt
        assert y2.tolist() == y.tolist()        # same per-row order


def test_two_stages_random_structures_within_tolerance():
    """The simulated method equals the plain definition within 1e-13 * scale
    on random structures with many empty rows and rows spanning many tiles."""
    cases = [
        synth.random_lengths(3000, seed=31, mean=6, p_empty=0.5),
        synth.random_lengths(2000, seed=32, mean=20, p_empty=0.05, p_long=0.002, long_len=5000),
        np.concatenate([np.zeros(50, int), [20000], np.zeros(70, int)]),
    ]
    for i, lens in enumerate(cases):
        A = synth.from_lengths(lens, 3000, seed=40 + i)
        x = synth.sym_vector(3000, seed=50 + i)
        yref, s = oracle.spmv_dot2(A.row_ptr, A.col, A.val, x)
        for T, W, S in [(32, 4, 7), (32, 16, 3), (8, 16, 6), (4, 6, 2), (32, 1, 1)]:
            st = oracle.speculative_stage(A.row_ptr, A.col, A.val, x, T, W, S)
            y = oracle.checking_stage(A.row_ptr, T, W, S, st)
            assert np.all(np.abs(y - yref) <= 1e-13 * s), (i, T, W, S)
            assert np.all(y[s == 0] == 0.0)


# ---------------------------------------------------------------------------
# the row loop restricted to a range of nonzeros (one shard of a split product)

def test_range_sums_on_the_6x6_example_by_hand():
    """Entries [4, 9) of the Sec. 2.1 example are e, f (row 1), g, h (row 2)
    and i (row 4): with x = (1..6) the partial rows are 2e+3f, 3g+5h, 5i."""
    g = _load("paper_example_6x6.json")
    sub = {s: float(3 + 2 * i) for i, s in enumerate(g["val_symbols"])}
    val = np.array([sub[s] for s in g["val_symbols"]])
    y = oracle.spmv_range(g["row_ptr"], g["col_idx"], val, np.array(g["x"], dtype=float), 4, 9)
    want = [0.0, 2 * sub["e"] + 3 * sub["f"], 3 * sub["g"] + 5 * sub["h"], 0.0, 5 * sub["i"], 0.0]
    assert y.tolist() == want
    # an empty range contributes nothing; the whole range is the plain product
    assert not oracle.spmv_range(g["row_ptr"], g["col_idx"], val, np.array(g["x"], float), 7,
                                 7).any()
    full = oracle.spmv_range(g["row_ptr"], g["col_idx"], val, np.array(g["x"], float), 0, 12)
    assert full.tolist() == [sum(c * sub[s] for s, c in co.items()) for co in g["y_coefficients"]]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_range_sums_add_up_to_the_product(seed):
    """Over any partition of [0, nnz) into ranges (cuts inside rows, at row
    starts, empty ranges) the range sums add up to the row loop's y exactly
    (small integers: every sum is exact in any order)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lens = rng.integers(0, 60, size=400)
    lens[rng.integers(0, 400, size=3)] = 3000       # rows over several cuts
    rp = np.zeros(401, np.int32)
    np.cumsum(lens, out=rp[1:])
    nnz = int(rp[-1])
    col = rng.integers(0, 90, size=nnz).astype(np.int32)
    val = rng.integers(-7, 8, size=nnz).astype(float)
    x = rng.integers(-7, 8, size=90).astype(float)
    cuts = np.unique(np.concatenate([[0, nnz], rng.integers(0, nnz + 1, size=9),
                                     rp[rng.integers(0, 401, size=3)]]))
    cuts = np.concatenate([cuts[:2], cuts[1:]])                  # one empty range too
    total = np.zeros(400)
    for B, E in zip(cuts[:-1], cuts[1:]):
        total += oracle.spmv_range(rp, col, val, x, int(B), int(E))
    assert np.array_equal(total, oracle.spmv(rp, col, val, x))
