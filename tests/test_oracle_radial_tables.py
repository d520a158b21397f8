"""Pins of the oracle's exact expansion tables against the two tables of the paper's appendix on the
compression of the radial expansion: the ranks of Table 3 and the worked exp(-r) example.

For a kernel with K' = q K, q a Laurent polynomial, every derivative is K^(m) = E(r) L_m(r) with
L_m a Laurent polynomial (L_{m+1} = L_m' + q L_m), so the degree-k radial part of the expansion,
    K^(k)_p(r', r) = sum_{j = k, k+2, ..., <= p} r'^j sum_{m <= j} K^(m)(r) r^(m-j) Tbar_{k,j,m},
is E(r) times a polynomial in r' and r (Theorem 3.1 with the tables of oracle/tables.py).  The
smallest number of separable terms F(r) G(r') is the rank of its coefficient matrix (rows: powers
of r', columns: powers of r), computed here exactly over the rationals.  Table 3 prints that rank
for eight kernels in d = 3..9; "-" means no compression (full rank).  The binomial factor of
eq. prelemma, the m = 0 term of the n-sum and every sign of the tables enter these ranks: dropping
either or flipping the m = 1 sign changes them (checked below).
"""
import os
from collections import defaultdict
from fractions import Fraction
from math import factorial

import pytest

from oracle import tables as T

HERE = os.path.dirname(os.path.abspath(__file__))
P = 12   # enough rows (7 at k = 0) for every printed rank
DIMS = [3, 4, 5, 6, 7, 8, 9]

# K = E(r) L_0(r), K' = q K: (L_0, q) as {power: coefficient}
KERNELS = {
    "1/r": ({-1: 1}, {}),                       # E = 1; K' = -K/r is carried by L_m' alone
    "1/r^2": ({-2: 1}, {}),
    "1/r^3": ({-3: 1}, {}),
    "exp(-r)/r": ({-1: 1}, {0: -1}),           # E = exp(-r)
    "exp(-r)": ({0: 1}, {0: -1}),
    "r*exp(-r)": ({1: 1}, {0: -1}),
    "exp(-1/r)": ({0: 1}, {-2: 1}),            # E = exp(-1/r), q = 1/r^2
    "exp(-1/r^2)": ({0: 1}, {-3: 2}),          # E = exp(-1/r^2), q = 2/r^3
}


def _table3():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "table3.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        rows[f[0]] = ([None if v == "-" else int(v) for v in f[1:8]], len(f) > 8 and f[8] == "unreproduced")
    return rows


def _derivs(name, n):
    L0, q = KERNELS[name]
    Ls = [{e: Fraction(c) for e, c in L0.items()}]
    for _ in range(n):
        L = Ls[-1]
        nxt = defaultdict(Fraction)
        for e, c in L.items():
            if e:
                nxt[e - 1] += c * e
            for e2, c2 in q.items():
                nxt[e + e2] += c * c2
        Ls.append({e: c for e, c in nxt.items() if c})
    return Ls


def _rank(rows):
    M = [list(r) for r in rows]
    rk = 0
    for c in range(len(M[0]) if M else 0):
        piv = next((i for i in range(rk, len(M)) if M[i][c] != 0), None)
        if piv is None:
            continue
        M[rk], M[piv] = M[piv], M[rk]
        for i in range(len(M)):
            if i != rk and M[i][c] != 0:
                f = M[i][c] / M[rk][c]
                M[i] = [a - f * b for a, b in zip(M[i], M[rk])]
        rk += 1
    return rk


def radial_rank(name, k, p, d, tbar=T.Tbar):
    """(rank, number of j rows) of the coefficient matrix of K^(k)_p(r', r) / E(r)."""
    Ls = _derivs(name, p)
    polys = []
    for j in range(k, p + 1, 2):
        poly = defaultdict(Fraction)
        for m in range(j + 1):
            t = tbar(k, j, m, d)
            if t:
                for e, c in Ls[m].items():
                    poly[e + m - j] += c * t
        polys.append(poly)
    cols = sorted({e for q in polys for e in q})
    return _rank([[q.get(e, Fraction(0)) for e in cols] for q in polys]), len(polys)


@pytest.mark.parametrize("name", [n for n, (_, unrep) in _table3().items() if not unrep])
def test_table3_radial_ranks(name):
    printed, _ = _table3()[name]
    for d, want in zip(DIMS, printed):
        for k in (0, 1):
            rank, rows = radial_rank(name, k, P, d)
            expect = rows if want is None else min(want, rows)
            assert rank == expect, (name, d, k, rank, want, rows)


def test_table3_rows_not_reproduced_are_full_rank():
    """exp(-1/r) and exp(-1/r^2): the exact tables give no compression at any d (printed: 4 and
    2); recorded as a reading, not a pin."""
    for name, (_, unrep) in _table3().items():
        if unrep:
            for d in (3, 4, 9):
                rank, rows = radial_rank(name, 0, P, d)
                assert rank == rows, (name, d)


def test_table3_catches_planted_table_mistakes():
    def no_binomial(k, j, m, d):          # the printed final formula, without the binomial
        if j < k or (j - k) % 2 or m < 0 or m > j:
            return Fraction(0)
        return sum((T.A(k, 2 * n - j, d) * Fraction(-2) ** (2 * n - j) * T.B(n, m) / factorial(n)
                    for n in range(max((j + k) // 2, m), j + 1)), Fraction(0))

    def no_m0(k, j, m, d):                # the sums of Theorem 3.1 as printed, from m = 1
        return Fraction(0) if m == 0 else T.Tbar(k, j, m, d)

    def flipped(k, j, m, d):
        v = T.Tbar(k, j, m, d)
        return -v if m == 1 else v

    assert radial_rank("exp(-r)", 0, P, 3, no_binomial)[0] != 2
    assert radial_rank("1/r", 0, P, 3, no_m0)[0] != 1
    assert radial_rank("exp(-r)", 0, P, 5, flipped)[0] != 3


def _exp_decomp():
    F, G = defaultdict(dict), defaultdict(dict)
    for line in open(os.path.join(HERE, "golden", "exp_decomp.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        poly = {int(t.split(":")[0]): Fraction(t.split(":")[1]) for t in f[3:]}
        (F if f[0] == "F" else G)[int(f[1])][int(f[2])] = poly
    return F, G


def radial_part_exp(k, p, tbar=T.Tbar):
    """{(power of r', power of r): coefficient} of the degree-k radial part of exp(-|r - r'|) in
    d = 3, divided by exp(-r): sum_j r'^j sum_m (-1)^m r^(m-j) Tbar_{k,j,m}."""
    out = defaultdict(Fraction)
    for j in range(k, p + 1, 2):
        for m in range(j + 1):
            t = tbar(k, j, m, 3)
            if t:
                out[(j, m - j)] += (-1) ** m * t
    return {key: v for key, v in out.items() if v}


@pytest.mark.parametrize("k", [0, 1, 2])
def test_exp_decomp_worked_example(k):
    """The printed F_{k,i} G_{k,i} of exp(-r), times r'^k / r^(k+1), equal the tables' radial part
    term by term, for every power of r' the table prints (up to r'^(k+6))."""
    F, G = _exp_decomp()
    printed = defaultdict(Fraction)
    for i in F[k]:
        for e, c in F[k][i].items():
            for j, g in G[k][i].items():
                printed[(j + k, e - k - 1)] += c * g
    printed = {key: v for key, v in printed.items() if v}
    jmax = max(j for j, _ in printed)
    ours = {key: v for key, v in radial_part_exp(k, jmax).items() if key[0] <= jmax}
    assert ours == printed


def test_exp_decomp_catches_the_printed_tbar_formula():
    """Without the binomial of eq. prelemma the k = 1 radial part no longer matches the worked example."""
    def no_binomial(k, j, m, d):
        if j < k or (j - k) % 2 or m < 0 or m > j:
            return Fraction(0)
        return sum((T.A(k, 2 * n - j, d) * Fraction(-2) ** (2 * n - j) * T.B(n, m) / factorial(n)
                    for n in range(max((j + k) // 2, m), j + 1)), Fraction(0))

    assert radial_part_exp(1, 7, no_binomial) != radial_part_exp(1, 7)
    assert radial_part_exp(1, 7, no_binomial)[(3, -1)] != Fraction(-1, 5)
