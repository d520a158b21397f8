"""The float64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer (host only).

The oracle is the checker every parity test trusts, so its C code is rebuilt with
-fsanitize=address,undefined (undefined behaviour aborts) and driven through its own Python
wrapper in a child process with the sanitizer runtimes preloaded: trees, s2m, traversal and the
dense product for d = 3 and 4, a singular kernel, and duplicate points.  Any out-of-bounds access,
use after free or undefined operation ends the child with a report and fails the test.
"""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    import numpy as np
    sys.path.insert(0, {root!r})
    from oracle import oracle as O
    O._SO = {so!r}
    O.build = lambda force=False: O._SO
    from paper_2106_04487_gb300 import inputs
    X = inputs.gaussian_mixture(3000, 3, 10, 0.05, seed=1)
    X[100:140] = X[99]                                   # duplicates: r = 0 pairs, oversize leaves
    W = inputs.normal_weights(3000, 3, seed=2).astype(np.float64)
    idx = np.arange(0, 3000, 7)
    for kern in ("matern32", "laplace", "ratquad"):
        kp = O.kparams(kern, 0.2, alpha=0.7)
        z = O.FKT(X, kp, p=5, leaf_size=32, theta=0.5).mvm(W, idx)
        zd = O.dense(X, kp, W, idx)
        assert np.linalg.norm(z - zd) < 1e-2 * np.linalg.norm(zd), kern
    X4 = inputs.gaussian_mixture(2000, 4, 10, 0.05, seed=3)
    z4 = O.FKT(X4, O.kparams("matern52", 0.3), p=4, leaf_size=64, theta=0.5).mvm(W[:, :2000], idx[idx < 2000])
    assert np.isfinite(z4).all()
    print("sanitized oracle ok")
""")


def test_oracle_clean_under_asan_and_ubsan(tmp_path):
    libs = []
    for name in ("libasan.so", "libubsan.so"):
        path = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
        if not os.path.isabs(path) or not os.path.exists(path):
            pytest.skip(f"{name} not available")
        libs.append(path)
    so = str(tmp_path / "liborc_san.so")
    subprocess.run(["gcc", "-O1", "-g", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer",
                    "-o", so, os.path.join(ROOT, "oracle", "fkt_oracle.c"), "-lm"], check=True)
    env = dict(os.environ, LD_PRELOAD=" ".join(libs), ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1", OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, so=so)], capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0 and "sanitized oracle ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
