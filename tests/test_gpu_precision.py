"""Precision form: the far-field contraction on the tensor cores (tcgen05.mma, float32
accumulation in tensor memory) with TF32, BF16 or BF16 hi/lo split operands, near field in
float32.  Each mode's error against the oracle FKT (float64) is checked against a stated bar."""
import numpy as np
import pytest

from paper_2106_04487_gb300 import inputs

pytestmark = pytest.mark.gpu

# Relative 2-norm error bars against the oracle FKT.  The hi/lo BF16 split drops only the lo*lo
# product (about 2^-16 per far term); TF32 keeps 10 mantissa bits, BF16 7.
BARS = {"bf16x3": 3e-5, "tf32": 2e-3, "bf16": 1e-2, "fp32": 1e-5}


@pytest.fixture(scope="module")
def fkt():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_04487_gb300 import build, fkt as F

    build.build()
    F.lib()
    return F


def _rel(a, b):
    return max(np.linalg.norm(a[i] - b[i]) / np.linalg.norm(b[i]) for i in range(len(b)))


@pytest.fixture(scope="module")
def case3(orc):
    X = inputs.gaussian_mixture(30000, 3, 10, 0.05, seed=40)
    W = inputs.normal_weights(30000, 40, seed=41)
    z = orc.FKT(X, orc.kparams("matern32", 0.2), p=6, leaf_size=128, theta=0.5).mvm(W)
    return X, W, z


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "bf16", "fp32"])
@pytest.mark.parametrize("nrhs", [1, 8, 40])
def test_precision_modes_d3(fkt, case3, prec, nrhs):
    import torch

    X, W, z = case3
    plan = fkt.Plan(torch.from_numpy(X).cuda(), "matern32", lengthscale=0.2, p=6, leaf_size=128, theta=0.5)
    plan.set_option("far_precision", prec)
    y = plan.mvm(torch.from_numpy(W[:nrhs]).cuda()).cpu().numpy().astype(np.float64)
    plan.check()
    err = _rel(y, z[:nrhs])
    print(f"d=3 {prec} nrhs={nrhs}: rel err vs oracle {err:.3e}")
    assert np.isfinite(y).all()
    assert err < BARS[prec], err


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "bf16"])
def test_precision_modes_d4(fkt, orc, prec):
    import torch

    X = inputs.gaussian_mixture(12000, 4, 20, 0.05, seed=42)
    W = inputs.normal_weights(12000, 10, seed=43)
    z = orc.FKT(X, orc.kparams("matern52", 0.3), p=5, leaf_size=128, theta=0.5).mvm(W)
    plan = fkt.Plan(torch.from_numpy(X).cuda(), "matern52", lengthscale=0.3, p=5, leaf_size=128, theta=0.5)
    plan.set_option("far_precision", prec)
    y = plan.mvm(torch.from_numpy(W).cuda()).cpu().numpy().astype(np.float64)
    plan.check()
    err = _rel(y, z)
    print(f"d=4 {prec}: rel err vs oracle {err:.3e}")
    assert err < BARS[prec], err
