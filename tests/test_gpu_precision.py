"""Precision form: the far-field contraction on the tensor cores (tcgen05.mma, float32
accumulation in tensor memory) with TF32, BF16 or BF16 hi/lo split operands, near field in
float32 -- on the CUDA cores, or as a TF32 hi/lo split product on the tensor cores (float32
kernel values, about 20 significant bits per product).  Each mode's error against the oracle
FKT (float64) is checked against a stated bar."""
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


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
@pytest.mark.parametrize("far_kernel", ["pairs", "single", "held"])
@pytest.mark.parametrize("p,nrhs", [(0, 8), (3, 13), (4, 8), (6, 40), (8, 32)])
def test_far_kernel_variants_d3(fkt, orc, prec, far_kernel, p, nrhs):
    """Both tensor-core far kernels (two far entries per thread in packed float32 pairs, or one)
    at several orders, including an odd number of entries per block and orders past the paired
    kernel's tensor-memory limit (which fall back to one entry per thread), against the oracle."""
    import torch

    X = inputs.gaussian_mixture(20000, 3, 10, 0.05, seed=49)
    W = inputs.normal_weights(20000, nrhs, seed=50)
    z = orc.FKT(X, orc.kparams("cauchy", 0.05), p=p, leaf_size=100, theta=0.5).mvm(W)
    plan = fkt.Plan(torch.from_numpy(X).cuda(), "cauchy", lengthscale=0.05, p=p, leaf_size=100, theta=0.5)
    plan.set_option("far_precision", prec)
    plan.set_option("far_kernel", far_kernel)
    y = plan.mvm(torch.from_numpy(W).cuda()).cpu().numpy().astype(np.float64)
    plan.check()
    err = _rel(y, z)
    print(f"far {prec} {far_kernel} p={p} nrhs={nrhs}: rel err vs oracle {err:.3e}")
    assert np.isfinite(y).all()
    assert err < BARS[prec], err


@pytest.mark.parametrize("kernel,ell,alpha", [("gaussian", 0.1, 1.0), ("exponential", 0.3, 1.0),
                                              ("matern52", 0.3, 1.0), ("ratquad", 0.2, 0.5), ("laplace", 1.0, 1.0)])
def test_far_pairs_every_kernel(fkt, orc, kernel, ell, alpha):
    """The packed-pair jets of every kernel kind (the paired kernel has its own recurrences)."""
    import torch

    X = inputs.gaussian_mixture(15000, 3, 10, 0.05, seed=51)
    W = inputs.normal_weights(15000, 32, seed=52)
    z = orc.FKT(X, orc.kparams(kernel, ell, alpha=alpha), p=5, leaf_size=128, theta=0.5).mvm(W)
    plan = fkt.Plan(torch.from_numpy(X).cuda(), kernel, lengthscale=ell, alpha=alpha, p=5, leaf_size=128, theta=0.5)
    plan.set_option("far_precision", "bf16x3")
    y = plan.mvm(torch.from_numpy(W).cuda()).cpu().numpy().astype(np.float64)
    plan.check()
    err = _rel(y, z)
    print(f"far pairs {kernel}: rel err vs oracle {err:.3e}")
    assert err < BARS["bf16x3"], err


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


# The tensor-core near field (32-wide passes) keeps the float32 bar: the hi/lo split leaves at most
# about 2^-20 of each product.
@pytest.mark.parametrize("near", ["tf32x3", "f16x3"])
@pytest.mark.parametrize("far", ["fp32", "bf16x3"])
@pytest.mark.parametrize("nrhs", [20, 32, 40])
def test_near_tensor_core_d3(fkt, case3, far, nrhs, near):
    import torch

    X, W, z = case3
    plan = fkt.Plan(torch.from_numpy(X).cuda(), "matern32", lengthscale=0.2, p=6, leaf_size=128, theta=0.5)
    plan.set_option("far_precision", far)
    plan.set_option("near_precision", near)
    y = plan.mvm(torch.from_numpy(W[:nrhs]).cuda()).cpu().numpy().astype(np.float64)
    plan.check()
    err = _rel(y, z[:nrhs])
    print(f"d=3 near {near}, far {far}, nrhs={nrhs}: rel err vs oracle {err:.3e}")
    assert np.isfinite(y).all()
    assert err < BARS[far], err


@pytest.mark.parametrize("kernel,ell,d,leaf", [("gaussian", 0.1, 3, 256), ("laplace", 1.0, 3, 64),
                                               ("cauchy", 0.05, 3, 200), ("exponential", 0.3, 3, 96),
                                               ("ratquad", 0.2, 3, 128), ("matern52", 0.3, 4, 128),
                                               ("gaussian", 0.2, 4, 77)])
@pytest.mark.parametrize("near", ["tf32x3", "f16x3"])
def test_near_tensor_core_kernels(fkt, orc, kernel, ell, d, leaf, near):
    """Every kernel kind, d = 3 and 4, ragged leaves (sizes not multiples of the 8-source MMA
    step), duplicated points (Laplace skips r = 0 pairs) against the oracle FKT."""
    import torch

    n = 9000
    X = inputs.gaussian_mixture(n, d, 10, 0.05, seed=44) if d == 3 else inputs.gaussian_mixture(n, d, 20, 0.05, seed=44)
    X[:50] = X[50:100]  # exact duplicates
    W = inputs.normal_weights(n, 32, seed=45)
    z = orc.FKT(X, orc.kparams(kernel, ell), p=4, leaf_size=leaf, theta=0.5).mvm(W)
    plan = fkt.Plan(torch.from_numpy(X).cuda(), kernel, lengthscale=ell, p=4, leaf_size=leaf, theta=0.5)
    plan.set_option("near_precision", near)
    y = plan.mvm(torch.from_numpy(W).cuda()).cpu().numpy().astype(np.float64)
    plan.check()
    err = _rel(y, z)
    print(f"{kernel} d={d} leaf={leaf} near {near}: rel err vs oracle {err:.3e}")
    assert err < BARS["fp32"], err


def test_near_f16_weight_ranges(fkt, orc):
    """The FP16 near field scales each right-hand side's weights by a power of two (its largest
    |w| into [2^13, 2^14)) and the kernel values by 2^14: right-hand sides from 1e-30 to 1e30 in
    size, an all-zero one and one with a single non-zero weight keep the float32 bar."""
    import torch

    X = inputs.gaussian_mixture(9000, 3, 10, 0.05, seed=53)
    W = inputs.normal_weights(9000, 32, seed=54).astype(np.float64)
    W *= np.logspace(-30, 30, 32)[:, None]
    W[3] = 0.0
    W[4] = 0.0
    W[4, 17] = 2.5
    W = W.astype(np.float32)
    z = orc.FKT(X, orc.kparams("gaussian", 0.1), p=4, leaf_size=128, theta=0.5).mvm(W)
    plan = fkt.Plan(torch.from_numpy(X).cuda(), "gaussian", lengthscale=0.1, p=4, leaf_size=128, theta=0.5)
    plan.set_option("near_precision", "f16x3")
    y = plan.mvm(torch.from_numpy(W).cuda()).cpu().numpy().astype(np.float64)
    plan.check()
    assert np.all(y[3] == 0.0)
    rows = [r for r in range(32) if r != 3]
    err = _rel(y[rows], z[rows])
    print(f"f16x3 weight ranges: rel err vs oracle {err:.3e}")
    assert err < BARS["fp32"], err


def test_near_tensor_core_all_near_matches_dense(fkt, orc):
    """One leaf holding every point (leaf_size >= N): the tensor-core near field alone is the
    dense product; compared with the float64 dense oracle."""
    import torch

    X = inputs.uniform_cube(3000, 3, seed=46)
    W = inputs.normal_weights(3000, 32, seed=47)
    z = orc.dense(X, orc.kparams("matern32", 0.2), W)
    plan = fkt.Plan(torch.from_numpy(X).cuda(), "matern32", lengthscale=0.2, p=4, leaf_size=4096, theta=0.5)
    plan.set_option("near_precision", "tf32x3")
    y = plan.mvm(torch.from_numpy(W).cuda()).cpu().numpy().astype(np.float64)
    plan.check()
    err = _rel(y, z)
    print(f"all-near tf32x3 vs dense float64: {err:.3e}")
    assert err < 2e-6, err


def test_near_precision_option_rejects_unknown(fkt):
    import torch

    X = inputs.uniform_cube(500, 3, seed=48)
    plan = fkt.Plan(torch.from_numpy(X).cuda(), "gaussian", lengthscale=0.1, p=2, leaf_size=64, theta=0.5)
    with pytest.raises(Exception):
        plan.set_option("near_precision", "bf16")
