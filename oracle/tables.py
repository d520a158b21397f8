"""Exact rational coefficient tables of the generalized multipole expansion.

TEST INFRASTRUCTURE ONLY.  This module is part of the CPU oracle: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it.  The GPU library computes its own tables by a different route and
never reads these.

Everything here is exact (``fractions.Fraction``) and follows the appendix
derivation of the paper (Sec. A.2, "Derivation of the FKT expansion"):

* ``A(k, i, d)``  -- change of basis cos^i = sum_k A_{k,i} C_k^alpha   (eq. coschange)
* ``B(n, m)``     -- Faa di Bruno coefficients of K(r sqrt(1+eps))       (Lemma A.2, eq. faa)
* ``Tbar(k,j,m,d)``-- radial coefficient table of Theorem 3.1 (eq. kdef),
  with the factor binom(n, 2n-j) that the binomial expansion in eq. prelemma
  carries.  The printed final formula omits it; with it the expansion
  reproduces the paper's Table 4 and collapses to the Legendre multipole for
  1/r (Sec. 3.3, eq. electro); without it the error grows with p.
* The n-sum starts at m = 0 with B_{0,0} = 1 (the theorem's printed sums start
  at m = 1), so the kernel value itself (n = 0 term of eq. taylor) is kept.
* The printed A_{k,i} denominator "(i-k)/2" is read as ((i-k)/2)!, which makes
  eq. coschange hold for d = 3 and 4.
* d = 2 (alpha = 0): C_k^0 vanishes for k >= 1, so the zonal functions are the limits
  C_k^alpha / alpha -> (2/k) T_k (Chebyshev) for k >= 1 and C_0 = T_0 = 1; the expansion is
  taken in T_k directly: cos^i = sum_k A_{k,i} T_k with A_{k,i} the alpha -> 0 limit of
  alpha (2/k) A_{k,i}(alpha) (k >= 1) and of A_{0,i}(alpha) (k = 0), and the 2-D addition
  theorem T_k(cos(phi - phi')) = cos k phi cos k phi' + sin k phi sin k phi'.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import comb, factorial


def alpha_of(d: int) -> Fraction:
    """Gegenbauer index alpha = d/2 - 1 (Sec. A.1)."""
    return Fraction(d - 2, 2)


def rising(a: Fraction, n: int) -> Fraction:
    """Rising factorial (a)_n = a (a+1) ... (a+n-1) (Sec. A.2, after eq. coschange)."""
    out = Fraction(1)
    for t in range(n):
        out *= a + t
    return out


def double_factorial(n: int) -> int:
    """n!! with the conventions (-1)!! = 0!! = 1."""
    out = 1
    while n > 1:
        out *= n
        n -= 2
    return out


@lru_cache(maxsize=None)
def A(k: int, i: int, d: int) -> Fraction:
    """cos^i(g) = sum_k A_{k,i} C_k^alpha(cos g)  (eq. coschange); for d = 2 the zonal
    functions are T_k and A_{k,i} is the alpha -> 0 limit stated in the module docstring:
    2^(1-i) binom(i, (i-k)/2) for k >= 1 and 2^(-i) binom(i, i/2) for k = 0.

    Zero unless 0 <= k <= i and k == i (mod 2).
    """
    if k < 0 or k > i or (i - k) % 2:
        return Fraction(0)
    if d == 2:
        # limit of alpha (2/k) i! (alpha+k) / (2^i ((i-k)/2)! (alpha)_((i+k)/2+1)), with
        # (alpha)_n ~ alpha (n-1)! as alpha -> 0
        return Fraction(factorial(i), 2 ** i * factorial((i - k) // 2) * factorial((i + k) // 2)) * (2 if k else 1)
    a = alpha_of(d)
    num = factorial(i) * (a + k)
    den = Fraction(2) ** i * factorial((i - k) // 2) * rising(a, (i + k) // 2 + 1)
    return num / den


@lru_cache(maxsize=None)
def B(n: int, m: int) -> Fraction:
    """d^n/de^n K(r sqrt(1+e)) at e=0 = sum_m B_{n,m} K^(m)(r) r^m  (Lemma A.2).

    B_{0,0} = 1, B_{n,0} = B_{0,m} = 0 otherwise.
    """
    if n == 0 and m == 0:
        return Fraction(1)
    if m < 1 or m > n:
        return Fraction(0)
    sign = -1 if (n + m) % 2 else 1
    return Fraction(sign * double_factorial(2 * n - 2 * m - 1) * comb(2 * n - m - 1, m - 1), 2 ** n)


@lru_cache(maxsize=None)
def Tbar(k: int, j: int, m: int, d: int) -> Fraction:
    """Radial coefficient of Theorem 3.1 in the Gegenbauer normalisation.

    K(|r'-r|) = sum_k C_k^alpha(cos g) sum_{j>=k} r'^j sum_{m=0}^j K^(m)(r) r^(m-j) Tbar_{k,j,m}

    Tbar_{k,j,m} = sum_{n=max((j+k)/2, m)}^{j} A_{k,2n-j} (-2)^(2n-j) binom(n, 2n-j) B_{n,m} / n!
    (end of Sec. A.2, with the binomial of eq. prelemma kept, which the printed final formula omits).
    """
    if j < k or (j - k) % 2 or m < 0 or m > j:
        return Fraction(0)
    out = Fraction(0)
    for n in range(max((j + k) // 2, m), j + 1):
        i = 2 * n - j
        out += A(k, i, d) * Fraction(-2) ** i * comb(n, i) * B(n, m) / factorial(n)
    return out


def harmonic_dim(k: int, d: int) -> int:
    """|H_k| = binom(k+d-1, k) - binom(k+d-3, k-2) (Sec. A.3); d = 2: 1, 2, 2, ..."""
    return comb(k + d - 1, k) - (comb(k + d - 3, k - 2) if k >= 2 else 0)


def expansion_terms(p: int, d: int):
    """The (k, j) index pairs kept by the order-p truncation (eq. finaltrunc).

    k <= p, j in {k, k+2, ...} with j <= p; the rank of the radial part of
    degree k is floor((p-k)/2)+1 (Sec. A.3).
    """
    return [(k, j) for k in range(p + 1) for j in range(k, p + 1, 2)]


def num_terms(p: int, d: int) -> int:
    """Size of the expansion, sum_k |H_k| (floor((p-k)/2)+1) (eq. num_multipoles)."""
    return sum(harmonic_dim(k, d) for k, _ in expansion_terms(p, d))


def tbar_array(p: int, d: int):
    """Dense float64 array T[k, j, m] of shape (p+1, p+1, p+1) for the C oracle."""
    import numpy as np

    T = np.zeros((p + 1, p + 1, p + 1), dtype=np.float64)
    for k, j in expansion_terms(p, d):
        for m in range(j + 1):
            T[k, j, m] = float(Tbar(k, j, m, d))
    return T
