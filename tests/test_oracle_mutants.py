"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one of them.

Each mutant is a one-token edit of oracle/pcc_oracle.c (a dropped term, a
wrong sign, a wrong index, a transposed operand, a strict instead of an
inclusive comparison), compiled to a temporary library on the CPU.  The
pins below are the same closed forms and exact brute forces as in
test_oracle_pins.py, run against the mutant; at least one must fail.
"""
import itertools
import json
import math
import os
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import build as obuild

MUTANTS = {
    "numerator_mean_dropped": ("s += (u[k] - mu) * (v[k] - mv);",
                               "s += (u[k] - mu) * (v[k]);"),
    "numerator_sign": ("s += (u[k] - mu) * (v[k] - mv);",
                       "s -= (u[k] - mu) * (v[k] - mv);"),
    "denominator_sqrt_dropped": ("return num / sqrt(ssq_u * ssq_v);",
                                 "return num / (ssq_u * ssq_v);"),
    "mean_divisor": ("double m = s / (double)l;",
                     "double m = s / (double)(l - 1);"),
    "pair_index_offset": ("return pairs_before_row(n, i) + (j - i - 1);",
                          "return pairs_before_row(n, i) + (j - i);"),
    "pair_row_count": ("return i * (2 * n - i - 1) / 2;",
                       "return i * (2 * n - i + 1) / 2;"),
    "perm_wrong_operand": ("s += (u[k] - mu) * (v[perm[k]] - mv);",
                           "s += (u[perm[k]] - mu) * (v[k] - mv);"),
    "pairs_transposed_means": (
        "double num = centred_dot(X + i * ldx, mean[i], X + j * ldx, mean[j],",
        "double num = centred_dot(X + i * ldx, mean[j], X + j * ldx, mean[i],"),
    "edges_strict": ("if (fabs(r) >= tau) /* NaN", "if (fabs(r) > tau) /* NaN"),
    "standardize_sqrt_dropped": (
        "Z[i * ldz + k] = bad ? 0.0 : (X[i * ldx + k] - m) / sqrt(q);",
        "Z[i * ldz + k] = bad ? 0.0 : (X[i * ldx + k] - m) / q;"),
    "perm_count_strict": ("c += (rk >= robs);", "c += (rk > robs);"),
    "diag_row_count": ("return y * (2 * n - y + 1) / 2;",
                       "return y * (2 * n - y - 1) / 2;"),
    "cross_index_column_major": ("return y * ncol + x;",
                                 "return x * nrow + y;"),
    "cross_wrong_stats": ("eq1(num, sx[i], sy[j]);\n        }",
                          "eq1(num, sx[i], sx[j]);\n        }"),
    "cross_search_strict": ("if (mid * ncol <= J)", "if (mid * ncol < J)"),
}


def _hadamard(k):
    H = np.array([[1.0]])
    for _ in range(k):
        H = np.block([[H, H], [H, -H]])
    return H


def _exact_r2(u, v):
    l = len(u)
    mu, mv = Fraction(sum(u), l), Fraction(sum(v), l)
    num = sum((Fraction(a) - mu) * (Fraction(b) - mv) for a, b in zip(u, v))
    su = sum((Fraction(a) - mu) ** 2 for a in u)
    sv = sum((Fraction(b) - mv) ** 2 for b in v)
    return num * num / (su * sv), (num > 0) - (num < 0)


def _pins(L):
    """Return the names of the pins that fail for library L."""
    failed = []
    rng = np.random.default_rng(5)

    def check(name, ok):
        if not ok:
            failed.append(name)

    # golden worked example, affine closed form, numpy.corrcoef
    check("golden", abs(oracle.pcc_pair([1, 2, 3, 4, 5], [2, 4, 5, 4, 5], L)
                        - (3 / 5) ** 0.5) <= 2e-16)
    u = rng.standard_normal(37)
    check("affine", abs(oracle.pcc_pair(u, -3 * u + 2, L) + 1) <= 1e-13)
    X = rng.standard_normal((12, 29)) + 3
    I, J = np.triu_indices(12, 1)
    r = oracle.pcc_pairs(X, I, J, L)
    check("corrcoef", np.max(np.abs(r - np.corrcoef(X)[I, J])) <= 1e-14)
    check("packed", np.allclose(oracle.pcc_upper(X, L), np.corrcoef(X)[I, J],
                                atol=1e-14, rtol=0))
    # exact rational brute force
    for _ in range(20):
        a = [int(t) for t in rng.integers(-9, 10, size=6)]
        b = [int(t) for t in rng.integers(-9, 10, size=6)]
        if len(set(a)) == 1 or len(set(b)) == 1:
            continue
        r2, sg = _exact_r2(a, b)
        got = oracle.pcc_pair(np.array(a, float), np.array(b, float), L)
        if abs(got - sg * math.sqrt(float(r2))) > 1e-15:
            failed.append("exact")
            break
    # numbering round trips
    ok = True
    for n in (5, 9):
        Jc = 0
        for i in range(n):
            for j in range(i + 1, n):
                ok &= oracle.pair_index(n, i, j, L) == Jc
                ok &= oracle.pair_coords(n, Jc, L) == (i, j)
                Jc += 1
        Jc = 0
        for y in range(n):
            for x in range(y, n):
                ok &= oracle.job_index_diag(n, y, x, L) == Jc
                ok &= oracle.job_coords_diag(n, Jc, L) == (y, x)
                Jc += 1
    check("numbering", ok)
    # standardize: unit norm + Eq. (6) == Eq. (1)
    Z, flag = oracle.standardize(X, L)
    check("standardize", np.max(np.abs((Z ** 2).sum(1) - 1)) <= 1e-14
          and np.max(np.abs((Z[I] * Z[J]).sum(1) - np.corrcoef(X)[I, J]))
          <= 1e-14)
    # planted edges at tau = 1 (exact +-1 pairs)
    H = _hadamard(3)[1:]
    E = np.vstack([H[0], 3 * H[0] - 7, -2 * H[0] + 1, H[1:]])
    ei, ej, _ = oracle.edges(E, 1.0, L=L)
    check("edges", set(zip(ei.tolist(), ej.tolist()))
          == {(0, 1), (0, 2), (1, 2)})
    # identity permutations count every k; a known exact permutation
    perms = np.tile(np.arange(29, dtype=np.int32), (3, 1))
    c, _, _ = oracle.perm_counts(X, perms, I, J, L=L)
    check("perm_identity", bool(np.all(c == 3)))
    uu = np.array([1.0, 7, 2, 9, 4, 3])
    pi = np.array([3, 0, 5, 1, 2, 4], dtype=np.int32)
    vv = np.empty(6)
    vv[pi] = 2 * uu + 1
    c, _, _ = oracle.perm_counts(np.vstack([uu, vv]), pi[None], [0], [1],
                                 L=L)
    check("perm_operand", c[0] == 1)
    # complete permutation test, l = 5
    l = 5
    allp = np.array(list(itertools.permutations(range(l))), dtype=np.int32)
    Y = np.vstack([rng.choice(1000, size=l, replace=False)
                   for _ in range(2)]).astype(float)
    c, _, _ = oracle.perm_counts(Y, allp, [0], [1], L=L)
    a, b = [int(t) for t in Y[0]], [int(t) for t in Y[1]]
    r2o, _ = _exact_r2(a, b)
    want = sum(_exact_r2(a, [b[s] for s in p])[0] >= r2o for p in allp)
    check("perm_complete", c[0] == want)
    # non-symmetric jobs (Eq. (7)-(8)): numbering and the corrcoef block
    ok = True
    for nrow, ncol in ((5, 3), (3, 5)):
        Jc = 0
        for y in range(nrow):
            for x in range(ncol):
                ok &= oracle.cross_job_index(nrow, ncol, y, x, L) == Jc
                ok &= oracle.cross_job_coords(nrow, ncol, Jc, L) == (y, x)
                Jc += 1
    check("cross_numbering", ok)
    Xa = rng.standard_normal((11, 23)) * 2 + 1
    Yb = rng.standard_normal((6, 23)) * 5 - 3
    check("cross_corrcoef", np.max(np.abs(
        oracle.cross_rows(Xa, Yb, L=L)
        - np.corrcoef(np.vstack([Xa, Yb]))[:11, 11:])) <= 1e-14)
    return failed


def test_unmutated_oracle_passes_all_pins():
    assert _pins(oracle.lib()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(obuild.SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new)
    path = tmp_path / "mutant.c"
    path.write_text(mutated)
    so = str(tmp_path / "libmutant.so")
    obuild.build(force=True, src=str(path), out=so)
    # a mutant may write out of bounds: run its pins in a separate process
    # (a crash there counts as caught)
    here = os.path.dirname(os.path.abspath(__file__))
    code = ("import sys, json; sys.path[:0] = [%r, %r]; "
            "import test_oracle_mutants as t, oracle; "
            "print(json.dumps(t._pins(oracle.lib(%r))))"
            % (here, os.path.dirname(here), so))
    proc = subprocess.run([sys.executable, "-c", code], capture_output=True,
                          text=True, timeout=300)
    if proc.returncode == 0:
        failed = json.loads(proc.stdout.strip().splitlines()[-1])
        assert failed, f"mutant {name} passed every pin"
