"""Pins of the FP64 oracle against facts the paper and mathematics fix.

None of these compares the oracle with itself: every expected value is a
closed form, an invariant, a hand-worked fixture (tests/golden), an exact
rational brute force, or an independent library routine (numpy.corrcoef).
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line)
    return rows


# ---------------------------------------------------------------- Eq. (1)

def test_worked_examples_golden():
    """Hand-worked Eq. (1) values (tests/golden/pcc_worked_examples.txt)."""
    for row in _read_golden("pcc_worked_examples.txt"):
        name, u, v, r = [s.strip() for s in row.split("|")]
        u = np.array([float(t) for t in u.split()])
        v = np.array([float(t) for t in v.split()])
        want = eval(r)  # expressions like (3/5)**0.5 written in the fixture
        got = oracle.pcc_pair(u, v)
        if math.isnan(want):
            assert math.isnan(got), name
        else:
            assert abs(got - want) <= 2e-16, (name, got, want)


def test_self_correlation_is_one():
    rng = np.random.default_rng(11)
    for l in (2, 3, 17, 128, 1000):
        u = rng.standard_normal(l) * 3 + 5
        assert abs(oracle.pcc_pair(u, u) - 1.0) <= 4e-16


def test_affine_closed_form():
    """r(u, a*u + b) = sign(a) for a != 0 (Eq. (1), numerator = a*S_u)."""
    rng = np.random.default_rng(12)
    for _ in range(50):
        l = int(rng.integers(2, 300))
        u = rng.standard_normal(l)
        a = rng.uniform(0.1, 10) * rng.choice([-1, 1])
        b = rng.uniform(-100, 100)
        r = oracle.pcc_pair(u, a * u + b)
        assert abs(r - math.copysign(1.0, a)) <= 1e-13


def test_bounded_and_symmetric():
    """|r| <= 1 (Section I) and r(u,v) = r(v,u) exactly."""
    rng = np.random.default_rng(13)
    X = rng.standard_normal((40, 33))
    X[5] = X[4] * -2.5 + 1  # an exact anti-correlated pair
    I, J = np.triu_indices(40, 1)
    r = oracle.pcc_pairs(X, I, J)
    rt = oracle.pcc_pairs(X, J, I)
    assert np.all(np.abs(r) <= 1.0 + 1e-15)
    assert np.array_equal(r, rt)


def _hadamard(k):
    H = np.array([[1.0]])
    for _ in range(k):
        H = np.block([[H, H], [H, -H]])
    return H


def test_orthogonal_centred_vectors_give_zero():
    """Rows of a Hadamard matrix without the constant row have zero mean and
    are pairwise orthogonal: r = 0 exactly (integer arithmetic)."""
    H = _hadamard(5)[1:]  # 31 x 32
    I, J = np.triu_indices(H.shape[0], 1)
    r = oracle.pcc_pairs(H, I, J)
    assert np.all(r == 0.0)
    # and unit self-correlation
    d = oracle.pcc_pairs(H, np.arange(31), np.arange(31))
    assert np.all(d == 1.0)


def test_invariances():
    """Eq. (1) is invariant under x -> alpha*x + beta (alpha > 0), flips sign
    for alpha < 0 on one side, and is invariant under a permutation of the
    samples applied to both vectors."""
    rng = np.random.default_rng(14)
    for _ in range(30):
        l = int(rng.integers(3, 200))
        u, v = rng.standard_normal(l), rng.standard_normal(l)
        r = oracle.pcc_pair(u, v)
        al, be = rng.uniform(0.01, 50), rng.uniform(-1e3, 1e3)
        assert abs(oracle.pcc_pair(al * u + be, v) - r) <= 1e-13
        assert abs(oracle.pcc_pair(u, -al * v + be) + r) <= 1e-13
        p = rng.permutation(l)
        assert abs(oracle.pcc_pair(u[p], v[p]) - r) <= 1e-14


def _exact_r2_sign(u, v):
    """Exact rational r^2 and sign of Eq. (1) for integer vectors."""
    l = len(u)
    mu = Fraction(sum(u), l)
    mv = Fraction(sum(v), l)
    num = sum((Fraction(a) - mu) * (Fraction(b) - mv) for a, b in zip(u, v))
    su = sum((Fraction(a) - mu) ** 2 for a in u)
    sv = sum((Fraction(b) - mv) ** 2 for b in v)
    if su == 0 or sv == 0:
        return None, 0
    return num * num / (su * sv), (num > 0) - (num < 0)


def test_exact_rational_bruteforce():
    """Brute force with exact rationals on tiny integer inputs, the square
    root taken only at the end (in FP64)."""
    rng = np.random.default_rng(15)
    for _ in range(300):
        l = int(rng.integers(2, 9))
        u = [int(t) for t in rng.integers(-20, 21, size=l)]
        v = [int(t) for t in rng.integers(-20, 21, size=l)]
        r2, sg = _exact_r2_sign(u, v)
        got = oracle.pcc_pair(np.array(u, float), np.array(v, float))
        if r2 is None:
            assert math.isnan(got)
            continue
        want = sg * math.sqrt(float(r2))
        assert abs(got - want) <= 1e-15, (u, v, got, want)


def test_numpy_corrcoef_matches():
    """numpy.corrcoef (an independent library routine for Eq. (1))."""
    rng = np.random.default_rng(16)
    X = rng.standard_normal((25, 41)) * rng.uniform(0.1, 10, (25, 1)) + 4
    C = np.corrcoef(X)
    I, J = np.triu_indices(25, 1)
    r = oracle.pcc_pairs(X, I, J)
    assert np.max(np.abs(r - C[I, J])) <= 1e-14


def test_zero_variance_gives_nan():
    X = np.array([[1.0, 2, 3, 4], [5.0, 5, 5, 5], [2.0, 1, 0, 7]])
    r = oracle.pcc_upper(X)
    # pairs (0,1) (0,2) (1,2)
    assert math.isnan(r[0]) and math.isnan(r[2]) and not math.isnan(r[1])


def test_catastrophic_offset_is_handled():
    """Eq. (2)-style one-pass forms cancel for large offsets; Eq. (1) as
    written (two passes) keeps r(u, u + c) = 1 even at an offset of 1e8."""
    rng = np.random.default_rng(17)
    u = rng.standard_normal(512)
    v = u + 1e-3 * rng.standard_normal(512)
    r0 = oracle.pcc_pair(u, v)
    r1 = oracle.pcc_pair(u + 1e8, v + 1e8)
    assert abs(r0 - r1) <= 1e-9


# --------------------------------------------------- numbering, Eq. (9)-(15)

def test_pair_numbering_golden():
    for row in _read_golden("bijection_n5_strict.txt"):
        J, i, j = (int(t) for t in row.split())
        assert oracle.pair_index(5, i, j) == J
        assert oracle.pair_coords(5, J) == (i, j)
    assert oracle.num_pairs(5) == 10


def test_job_numbering_diag_golden():
    for row in _read_golden("bijection_n4_diag.txt"):
        J, y, x = (int(t) for t in row.split())
        assert oracle.job_index_diag(4, y, x) == J
        assert oracle.job_coords_diag(4, J) == (y, x)


def test_pair_numbering_exhaustive():
    """The paper's own check (Section III-B): walk every coordinate in the
    sequential order, compare its computed id with the running count, and
    invert it back."""
    for n in list(range(2, 80)) + [255, 256, 257]:
        J = 0
        for i in range(n):
            for j in range(i + 1, n):
                assert oracle.pair_index(n, i, j) == J
                assert oracle.pair_coords(n, J) == (i, j)
                J += 1
        assert J == oracle.num_pairs(n) == n * (n - 1) // 2
        assert oracle.pair_index(n, 0, 0) == -1
        assert oracle.pair_index(n, 1, 0) == -1
        assert oracle.pair_index(n, 0, n) == -1


def test_job_numbering_diag_exhaustive():
    for n in range(1, 70):
        J = 0
        for y in range(n):
            for x in range(y, n):
                assert oracle.job_index_diag(n, y, x) == J
                assert oracle.job_coords_diag(n, J) == (y, x)
                J += 1
        assert J == n * (n + 1) // 2


def test_pair_numbering_large_rows():
    """Row starts and ends for large n (where float formulas break)."""
    for n in (65536, 65537, 1 << 20, 3_000_001):
        for i in list(range(0, 5)) + list(range(n - 6, n - 1)) + [n // 2,
                                                                 n // 3]:
            J0 = oracle.pair_index(n, i, i + 1)
            J1 = oracle.pair_index(n, i, n - 1)
            assert J0 == i * (2 * n - i - 1) // 2
            assert J1 - J0 == n - 2 - i
            assert oracle.pair_coords(n, J0) == (i, i + 1)
            assert oracle.pair_coords(n, J1) == (i, n - 1)


# ------------------------------------------------------- packed all-pairs

def test_packed_rows_match_pairs():
    rng = np.random.default_rng(18)
    X = rng.standard_normal((37, 19))
    R = oracle.pcc_upper(X)
    I, J = np.triu_indices(37, 1)  # row-major order == the numbering
    assert R.size == 37 * 36 // 2
    assert np.array_equal(R, oracle.pcc_pairs(X, I, J))
    # a middle row block
    sub = oracle.pcc_rows(X, 10, 20)
    a = oracle.pair_index(37, 10, 11)
    assert np.array_equal(sub, R[a:a + sub.size])


# -------------------------------------------------------------- Eq. (5)-(6)

def test_standardize_unit_norm_and_eq6():
    """Eq. (5) rows have zero sum and unit norm, and Eq. (6) (dot product of
    standardized rows) reproduces Eq. (1)."""
    rng = np.random.default_rng(19)
    X = rng.standard_normal((30, 50)) * 5 + 100
    X[7] = 3.0  # constant row
    Z, flag = oracle.standardize(X)
    assert flag.tolist() == [int(i == 7) for i in range(30)]
    ok = flag == 0
    assert np.max(np.abs(Z[ok].sum(1))) <= 1e-13
    assert np.max(np.abs((Z[ok] ** 2).sum(1) - 1)) <= 1e-14
    assert np.all(Z[7] == 0)
    I, J = np.triu_indices(30, 1)
    r = oracle.pcc_pairs(X, I, J)
    good = ok[I] & ok[J]
    eq6 = np.einsum("pk,pk->p", Z[I[good]], Z[J[good]])
    assert np.max(np.abs(eq6 - r[good])) <= 1e-14
    # exact-rational check of one standardized row (integer data)
    u = [3, 1, 4, 1, 5, 9, 2, 6]
    Zu, _ = oracle.standardize(np.array([u], float))
    m = Fraction(sum(u), len(u))
    s = sum((Fraction(a) - m) ** 2 for a in u)
    for k, a in enumerate(u):
        want = float(Fraction(a) - m) / math.sqrt(float(s))
        assert abs(Zu[0, k] - want) <= 1e-16


# ------------------------------------------------------------------- edges

def test_edges_planted_exact():
    """Rows 0-3 are exact affine copies of one Hadamard row (r = +-1
    exactly), the other Hadamard rows are orthogonal to it and to each
    other (r = 0): the |r| >= tau edge set is known in closed form for
    every tau in (0, 1]."""
    H = _hadamard(3)[1:]  # 7 x 8, zero-mean, orthogonal, entries +-1
    base = H[0]
    X = np.vstack([base, 3 * base - 7, -2 * base + 1, 0.5 * base + 2, H[1:]])
    for tau in (1.0, 0.8, 1e-9):
        I, J, r = oracle.edges(X, tau)
        got = set(zip(I.tolist(), J.tolist()))
        want = {(i, j) for i in range(4) for j in range(i + 1, 4)}
        assert got == want, tau
        sign = {(0, 1): 1, (0, 2): -1, (0, 3): 1, (1, 2): -1, (1, 3): 1,
                (2, 3): -1}
        for i, j, rv in zip(I, J, r):
            assert rv == sign[(int(i), int(j))]
    I, J, r = oracle.edges(X, 1.0, 1, 3)  # row range [1, 3)
    assert set(zip(I.tolist(), J.tolist())) == {(1, 2), (1, 3), (2, 3)}


def test_edges_never_include_nan_pairs():
    X = np.array([[1.0, 2, 3], [1.0, 2, 3], [4.0, 4, 4]])
    I, J, r = oracle.edges(X, 0.5)
    assert list(zip(I, J)) == [(0, 1)]


# ------------------------------------------------------- permutation test

def test_perm_identity_counts_all():
    rng = np.random.default_rng(20)
    X = rng.standard_normal((12, 16))
    P = 7
    perms = np.tile(np.arange(16, dtype=np.int32), (P, 1))
    I, J = np.triu_indices(12, 1)
    c, clo, chi = oracle.perm_counts(X, perms, I, J, delta=1e-9)
    assert np.all(c == P) and np.all(chi == P)


def test_perm_complete_test_exact():
    """Complete permutation test for l = 5 (all 120 permutations) against
    exact rational brute force on integer data with distinct values: only
    the identity ties exactly with r_obs, so the count is exact."""
    rng = np.random.default_rng(21)
    l = 5
    perms = np.array(list(itertools.permutations(range(l))), dtype=np.int32)
    for _ in range(12):
        X = np.vstack([rng.choice(10**6, size=l, replace=False)
                       for _ in range(4)]).astype(float)
        I, J = np.triu_indices(4, 1)
        c, _, _ = oracle.perm_counts(X, perms, I, J)
        for p, (i, j) in enumerate(zip(I, J)):
            u = [int(t) for t in X[i]]
            v = [int(t) for t in X[j]]
            r2obs, _ = _exact_r2_sign(u, v)
            want = 0
            for pi in perms:
                r2k, _ = _exact_r2_sign(u, [v[s] for s in pi])
                want += r2k >= r2obs
            assert c[p] == want, (p, c[p], want)


def test_perm_permutes_second_operand_only():
    """r_k(i,j) uses x_i as is and x_j read through pi_k: a permutation that
    maps x_j onto a scaled copy of x_i gives |r_k| = 1."""
    l = 6
    u = np.array([1.0, 7, 2, 9, 4, 3])
    pi = np.array([3, 0, 5, 1, 2, 4], dtype=np.int32)
    v = np.empty(l)
    v[pi] = 2 * u + 1  # so v[pi[s]] = 2u[s] + 1
    X = np.vstack([u, v])
    c, clo, chi = oracle.perm_counts(X, pi[None, :], [0], [1], delta=1e-12)
    assert c[0] == 1
    # the reverse convention (permuting x_i) would not give |r| = 1
    assert abs(oracle.pcc_pair(u[pi], v)) < 0.999


def test_perm_band_counts_bracket():
    rng = np.random.default_rng(22)
    X = rng.standard_normal((10, 24))
    perms = np.stack([rng.permutation(24) for _ in range(50)]).astype(np.int32)
    I, J = np.triu_indices(10, 1)
    c, clo, chi = oracle.perm_counts(X, perms, I, J, delta=0.05)
    assert np.all(clo <= c) and np.all(c <= chi)
    assert np.any(clo < chi)


# ------------------------------------------------- non-symmetric (cross)


def test_cross_job_numbering_exhaustive():
    # Eq. (7)-(8): row-major numbering of an nrow x ncol job matrix and its
    # inverse, every job of several ragged shapes
    for nrow, ncol in ((1, 1), (1, 7), (7, 1), (5, 3), (3, 5), (9, 13)):
        J = 0
        for y in range(nrow):
            for x in range(ncol):
                assert oracle.cross_job_index(nrow, ncol, y, x) == J
                assert oracle.cross_job_coords(nrow, ncol, J) == (y, x)
                J += 1
        assert oracle.cross_job_index(nrow, ncol, nrow, 0) == -1
        assert oracle.cross_job_index(nrow, ncol, 0, ncol) == -1
        with pytest.raises(ValueError):
            oracle.cross_job_coords(nrow, ncol, nrow * ncol)


def test_cross_matches_corrcoef_block():
    # the off-diagonal block of numpy.corrcoef over the stacked rows
    rng = np.random.default_rng(21)
    X = rng.standard_normal((11, 37)) * 3 + 5
    Y = rng.standard_normal((6, 37)) - 2
    R = oracle.cross_rows(X, Y)
    C = np.corrcoef(np.vstack([X, Y]))[:11, 11:]
    assert R.shape == (11, 6)
    assert np.max(np.abs(R - C)) <= 1e-14


def test_cross_closed_forms_and_bruteforce():
    # r(x_i, a x_i + b) = sign(a) placed at known (i, j); exact rationals
    rng = np.random.default_rng(22)
    X = rng.standard_normal((4, 19))
    Y = np.vstack([rng.standard_normal(19), -2.5 * X[2] + 1, 4 * X[0] - 3])
    R = oracle.cross_rows(X, Y)
    assert abs(R[2, 1] + 1) <= 1e-14 and abs(R[0, 2] - 1) <= 1e-14
    for _ in range(15):
        a = [int(t) for t in rng.integers(-9, 10, size=7)]
        b = [int(t) for t in rng.integers(-9, 10, size=7)]
        if len(set(a)) == 1 or len(set(b)) == 1:
            continue
        r2, sg = _exact_r2_sign(a, b)
        got = oracle.cross_rows(np.array([a], float), np.array([b], float))
        assert abs(got[0, 0] - sg * math.sqrt(float(r2))) <= 1e-15


def test_cross_rows_slices_and_pairs_agree():
    # rows [i0, i1) are the same numbers as the whole matrix's rows, and the
    # pair list gives the same value at every (i, j); swapping X and Y
    # transposes the result (Eq. (1) is symmetric in its operands)
    rng = np.random.default_rng(23)
    X = rng.random((9, 24))
    Y = rng.random((14, 24))
    R = oracle.cross_rows(X, Y)
    assert np.array_equal(oracle.cross_rows(X, Y, 3, 7), R[3:7])
    I, J = np.meshgrid(np.arange(9), np.arange(14), indexing="ij")
    assert np.array_equal(oracle.cross_pairs(X, Y, I.ravel(), J.ravel()),
                          R.ravel())
    assert np.array_equal(oracle.cross_rows(Y, X), R.T)
    assert np.array_equal(np.isnan(oracle.cross_rows(
        np.vstack([X, np.full(24, 2.0)]), Y))[9], np.ones(14, bool))
