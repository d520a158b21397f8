"""The library's expansion tables (row A6, host code in csrc/tables.cpp) against the oracle's exact
rational tables, on the CPU.

csrc/tables.cpp builds That_{k,j,m} = m! Tbar_{k,j,m} by composing power series and inverting the
Gegenbauer coefficient matrix; oracle/tables.py evaluates the appendix's closed forms in exact
rationals (pinned to Table 4, Table 3 and the worked exp(-r) example).  A small host harness
compiled with g++ from the library's own source prints every coefficient the kernels read for
d = 3 (p <= 10) and d = 4 (p <= 8); they must equal the exact values to float32 rounding.  The
build step also checks the addition theorem of its harmonic recurrences and must return FKT_OK.
"""
import os
import shutil
import subprocess
from math import factorial

import pytest

from oracle import tables as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2106_04487_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdlib>
#include "fkt_internal.h"
int main(int argc, char** argv) {
    const int d = atoi(argv[1]), p = atoi(argv[2]);
    fkt::FarTables t;
    const int rc = fkt::build_far_tables(d, p, &t);
    printf("rc %d\n", rc);
    int q = 0;
    for (int k = 0; k <= p; ++k)
        for (int j = k; j <= p; j += 2, ++q)
            for (int m = 0; m <= j; ++m) printf("%d %d %d %.9e\n", k, j, m, (double)t.That[q][m]);
    return 0;
}
"""


def _cuda_include():
    for c in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return os.path.join(c, "include")
    return None


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("g++ or the CUDA headers are missing")
    tmp = tmp_path_factory.mktemp("tables")
    src = tmp / "harness.cpp"
    src.write_text(HARNESS)
    exe = tmp / "harness"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-I", inc, str(src), os.path.join(CSRC, "tables.cpp"),
                    "-o", str(exe), "-lm"], check=True)
    return str(exe)


@pytest.mark.parametrize("d,p", [(3, 4), (3, 6), (3, 10), (4, 6), (4, 8)])
def test_library_tables_equal_the_exact_tables(harness, d, p):
    out = subprocess.run([harness, str(d), str(p)], capture_output=True, text=True, check=True).stdout.split("\n")
    assert out[0] == "rc 0"          # the harmonic recurrences passed the addition-theorem self-check
    rows = [ln.split() for ln in out[1:] if ln.strip()]
    assert len(rows) == sum(j + 1 for k in range(p + 1) for j in range(k, p + 1, 2))
    scale = max(abs(float(T.Tbar(int(k), int(j), int(m), d)) * factorial(int(m))) for k, j, m, _ in rows)
    for k, j, m, v in rows:
        k, j, m = int(k), int(j), int(m)
        exact = float(T.Tbar(k, j, m, d) * factorial(m))
        assert abs(float(v) - exact) <= 2e-7 * abs(exact) + 1e-12 * scale, (d, p, k, j, m, float(v), exact)


@pytest.mark.parametrize("p", [4, 8, 10])
def test_laplace_radial_terms_beyond_j_equal_k_vanish(harness, p):
    """The library keeps only the j = k terms for 1/r in d = 3 (its radial compression).  For that
    kernel J_m = K^(m)(r) r^m / m! = (-1)^m / r, so the degree-k, order-j radial function is
    R_kj(r) = (1/r) sum_m That_kjm (-1)^m: it must vanish for every j > k (rank 1 per degree,
    Table 3) -- exactly in the oracle's rationals and to float32 rounding in the library's tables --
    and not for j = k (the Legendre multipole r'^k / r^(k+1))."""
    from fractions import Fraction

    out = subprocess.run([harness, "3", str(p)], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [ln.split() for ln in out[1:] if ln.strip()]
    lib, ref, mag = {}, {}, {}
    for k, j, m, v in rows:
        k, j, m = int(k), int(j), int(m)
        lib[(k, j)] = lib.get((k, j), 0.0) + (-1) ** m * float(v)
        mag[(k, j)] = mag.get((k, j), 0.0) + abs(float(v))
        ref[(k, j)] = ref.get((k, j), Fraction(0)) + (-1) ** m * T.Tbar(k, j, m, 3) * factorial(m)
    for (k, j), s in ref.items():
        if j > k:
            assert s == 0, (k, j, s)
            assert abs(lib[(k, j)]) <= 1e-6 * mag[(k, j)], (k, j, lib[(k, j)], mag[(k, j)])
        else:
            assert s == 1, (k, j, s)             # Legendre normalisation: r'^k P_k(cos) / r^(k+1)
