"""Radial compression (the paper's appendix on compressing the radial expansion, Table 3): for the
Laplace kernel 1/r in d = 3 each degree-k radial part has rank 1 -- it is r'^k / r^(k+1) alone --
so the library drops the terms j > k from s2m, the multipoles and m2t ((p+1)^2 terms instead of
binom(p+3, 3): 49 of 84 at p = 6, 81 of 165 at p = 8).  The compressed product is the same
expansion, so it must match the uncompressed oracle FKT at the usual bars, on every far path."""
import numpy as np
import pytest

from bars import assert_bars
from paper_2106_04487_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fkt():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_04487_gb300 import build, fkt as F

    build.build()
    F.lib()
    return F


BARS = {"fp32": 1e-5, "bf16x3": 3e-5, "tf32": 2e-3, "bf16": 1e-2}


@pytest.mark.parametrize("p,far,nrhs", [(0, "fp32", 1), (3, "fp32", 8), (6, "fp32", 1), (6, "bf16x3", 32),
                                        (8, "bf16x3", 11), (8, "bf16", 4), (10, "fp32", 3), (10, "bf16x3", 8),
                                        (6, "tf32", 8)])
def test_compressed_laplace_matches_oracle(fkt, orc, p, far, nrhs):
    import torch

    X = inputs.uniform_plus_clusters(30000, 3, 20, 0.01, seed=81)
    W = inputs.uniform_weights(30000, nrhs, seed=82)
    scale = 1.0 / (4 * np.pi)
    plan = fkt.Plan(torch.from_numpy(X).cuda(), "laplace", lengthscale=1.0, scale=scale, p=p, leaf_size=128,
                    theta=0.5)
    assert plan.stats()["nterms"] == (p + 1) ** 2          # compressed by default
    plan.set_option("far_precision", far)
    Wd = torch.from_numpy(W).cuda()
    y = plan.mvm(Wd).cpu().numpy().astype(np.float64)
    plan.check()
    z = orc.FKT(X, orc.kparams("laplace", 1.0, scale=scale), p=p, leaf_size=128, theta=0.5).mvm(W)
    e2, einf = assert_bars(y, z, BARS[far], f"compressed laplace p={p} {far}")
    # the uncompressed layout on the same plan gives the same product (at p = 10 the BF16 hi/lo
    # operands of the 286-term full expansion exceed the tensor-core kernels' on-chip memory:
    # only the compressed 121-term expansion runs there)
    plan.set_option("radial_compression", "off")
    assert plan.stats()["nterms"] == (p + 1) * (p + 2) * (p + 3) // 6
    if p == 10 and far == "bf16x3":
        with pytest.raises(fkt.FktError):
            plan.mvm(Wd)
    else:
        y_full = plan.mvm(Wd).cpu().numpy().astype(np.float64)
        plan.check()
        assert_bars(y_full, z, BARS[far], f"uncompressed laplace p={p} {far}")
    plan.set_option("radial_compression", "auto")
    assert plan.stats()["nterms"] == (p + 1) ** 2
    print(f"laplace p={p} {far} nrhs={nrhs}: compressed vs oracle {e2:.2e} / {einf:.2e}")


def test_compression_only_where_exact(fkt):
    import torch

    X = torch.from_numpy(inputs.uniform_cube(2000, 3)).cuda()
    for kernel in ("gaussian", "matern32", "cauchy"):
        plan = fkt.Plan(X, kernel, lengthscale=0.2, p=6, leaf_size=128, theta=0.5)
        assert plan.stats()["nterms"] == 84
        plan.set_option("radial_compression", "auto")
        assert plan.stats()["nterms"] == 84
        plan.close()
    X4 = torch.from_numpy(inputs.uniform_cube(2000, 4)).cuda()
    plan = fkt.Plan(X4, "laplace", lengthscale=1.0, p=4, leaf_size=128, theta=0.5)
    assert plan.stats()["nterms"] == 70                    # 1/r in d = 4 has full radial rank
    with pytest.raises(fkt.FktError):
        plan.set_option("radial_compression", "on")
