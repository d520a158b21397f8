"""The headline benchmark configuration itself, at full size, in the launch configuration that
bench.py times, against the float64 oracle FKT (Algorithm 1, Theorem 3.1 / eq. finaltrunc).

Configuration: N = 1,000,000 points from the 10-component isotropic Gaussian mixture (centres
U[0,1]^3, std 0.05), Matern-3/2 l = 0.2 and Cauchy l = 0.05, p = 6, theta = 0.375, leaf 256,
32 right-hand sides N(0,1) in one pass, near field on the tensor cores with TF32 hi/lo operands,
far field on the tensor cores with BF16 hi/lo operands (float32 kernel values and accumulation).

At this size the tensor-core kernels run with several CTAs per SM, walk long interaction lists
through their 32-entry windows and flush their accumulators every few chunks or entries; these
tests pin exactly that path.  Sampled targets: 300 uniformly drawn, plus targets in partly-active
warps (an entry of their block taken by some but not all of their 32-target group, far and near
entries alike), half inside the entry's mask and half outside.  Bars: the bf16x3 far form's
3e-5, both per right-hand side (relative 2-norm) and per target (max |y - z| / |z|_inf).
"""
import numpy as np
import pytest

from bars import assert_bars, partly_masked_targets
from paper_2106_04487_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 3e-5   # BF16 hi/lo far field (three products per term, about 16 significant bits)
N, NRHS = 1_000_000, 32


@pytest.fixture(scope="module")
def fkt():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_04487_gb300 import build, fkt as F

    build.build()
    F.lib()
    return F


@pytest.fixture(scope="module")
def headline_inputs():
    # the same recipes and seeds as bench.py's default workload
    return inputs.gaussian_mixture(N, 3, 10, 0.05), inputs.normal_weights(N, NRHS)


@pytest.mark.parametrize("kernel,ell", [("matern32", 0.2), ("cauchy", 0.05)])
def test_headline_config_against_oracle_fkt(fkt, orc, headline_inputs, kernel, ell):
    import torch

    X, W = headline_inputs
    plan = fkt.Plan(torch.from_numpy(X).cuda(), kernel, lengthscale=ell, p=6, leaf_size=256, theta=0.375)
    plan.set_option("near_precision", "tf32x3")
    plan.set_option("far_precision", "bf16x3")
    Wd = torch.from_numpy(W).cuda()
    y = plan.mvm(Wd).cpu().numpy().astype(np.float64)
    plan.check()
    perm = plan.tree()["perm"]
    masked = partly_masked_targets(plan.lists(), 300, seed=11)
    plan.close()
    assert len(masked) >= 100, len(masked)
    idx = np.unique(np.concatenate([inputs.subsample(N, 300), perm[masked]]))
    z = orc.FKT(X, orc.kparams(kernel, ell), p=6, leaf_size=256, theta=0.375).mvm(W, idx)
    e2, einf = assert_bars(y[:, idx], z, TOL, f"{kernel} headline")
    print(f"{kernel}: {len(idx)} targets ({len(masked)} in partly-active warps): "
          f"rel 2-norm {e2:.2e}, element-wise {einf:.2e}")
    # the targets of partly-active warps on their own
    sub = np.searchsorted(idx, perm[masked])
    assert_bars(y[:, idx[sub]], z[:, sub], TOL, f"{kernel} partly-active warps")
