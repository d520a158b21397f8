"""GPU path (through the C ABI) against the CPU float64 oracle.

Bars: tree and interaction lists bit-identical to the oracle's (integer/index
work, float64 centres and radii); FKT output within relative 2-norm 1e-5 of the
oracle FKT on the same inputs (float32 arithmetic against float64).
"""
import numpy as np
import pytest

from bars import assert_bars
from paper_2106_04487_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fkt():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_04487_gb300 import build, fkt as F

    build.build()
    F.lib()
    return F


def _plan(fkt, X, kernel, ell, p, leaf, theta, alpha=1.0, scale=1.0):
    import torch

    return fkt.Plan(torch.from_numpy(X).cuda(), kernel, lengthscale=ell, alpha=alpha, scale=scale, p=p,
                    leaf_size=leaf, theta=theta)


def _gpu_mvm(plan, w):
    import torch

    return plan.mvm(torch.from_numpy(w).cuda()).cpu().numpy().astype(np.float64)


def _rel(a, b):
    a, b = np.atleast_2d(a), np.atleast_2d(b)
    return max(np.linalg.norm(a[i] - b[i]) / np.linalg.norm(b[i]) for i in range(len(b)))


def _oracle(orc, X, kernel, ell, p, leaf, theta, alpha=1.0, scale=1.0):
    return orc.FKT(X, orc.kparams(kernel, ell, alpha=alpha, scale=scale), p=p, leaf_size=leaf, theta=theta)


# ------------------------------------------------------------ tree & lists
@pytest.mark.parametrize("case", ["uniform", "gmm", "ball", "dups", "d4"])
def test_tree_identical_to_oracle(fkt, orc, case):
    X = {"uniform": lambda: inputs.uniform_cube(20000, 3),
         "gmm": lambda: inputs.gaussian_mixture(30000, 3, 10, 0.05),
         "ball": lambda: inputs.unit_ball(15000, 3),
         "dups": lambda: np.repeat(inputs.uniform_cube(50, 3, seed=3), 40, axis=0),
         "d4": lambda: inputs.gaussian_mixture(12000, 4, 20, 0.05)}[case]()
    leaf = 64 if case == "dups" else 256
    plan = _plan(fkt, X, "gaussian", 0.1, 4, leaf, 0.5)
    g = plan.tree()
    o = _oracle(orc, X, "gaussian", 0.1, 4, leaf, 0.5).tree()
    for k in ("perm", "begin", "end", "level", "leaf", "child"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    np.testing.assert_array_equal(g["centre"], o["centre"])
    np.testing.assert_array_equal(g["rho2"], o["rho2"])


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.75])
def test_lists_identical_to_oracle(fkt, orc, theta):
    """Per target: the far node set and the near leaf set equal the oracle's traversal (eq. accparam)."""
    X = inputs.gaussian_mixture(6000, 3, 5, 0.08, seed=1)
    plan = _plan(fkt, X, "matern32", 0.2, 4, 64, theta)
    ora = _oracle(orc, X, "matern32", 0.2, 4, 64, theta)
    perm = plan.tree()["perm"]
    far, near = plan.target_sets()
    rng = np.random.default_rng(0)
    for t in rng.choice(len(X), 400, replace=False):
        of, on = ora.target_lists(int(perm[t]))
        assert sorted(far[t]) == sorted(of.tolist()), t
        assert sorted(near[t]) == sorted(on.tolist()), t
    s = plan.stats()
    assert s["far_pairs"] == sum(len(v) for v in far.values())


# ------------------------------------------------------------------- MVM
def test_config_gaussian_20k(fkt, orc):
    """Uniform cube, Gaussian l=0.1, d=3, N=20,000, p=4, leaf 512, theta=0.5, one RHS."""
    X = inputs.uniform_cube(20000, 3)
    w = inputs.normal_weights(20000)
    y = _gpu_mvm(_plan(fkt, X, "gaussian", 0.1, 4, 512, 0.5), w)
    z = _oracle(orc, X, "gaussian", 0.1, 4, 512, 0.5).mvm(w)
    assert _rel(y, z) < TOL
    zd = orc.dense(X, orc.kparams("gaussian", 0.1), w)
    # against the dense product the GPU is as accurate as the expansion itself
    assert abs(_rel(y, zd) - _rel(z, zd)) < 1e-5


@pytest.mark.parametrize("kernel,ell,alpha,scale", [
    ("gaussian", 0.1, 1.0, 1.0), ("exponential", 0.3, 1.0, 1.0), ("matern32", 0.2, 1.0, 1.0),
    ("matern52", 0.3, 1.0, 2.0), ("cauchy", 0.05, 1.0, 1.0), ("ratquad", 0.2, 1.0, 1.0),
    ("ratquad", 0.2, 0.5, 1.0), ("laplace", 1.0, 1.0, 1.0 / (4 * np.pi))])
def test_kernels_d3(fkt, orc, kernel, ell, alpha, scale):
    X = inputs.gaussian_mixture(9000, 3, 6, 0.07, seed=4)
    w = inputs.normal_weights(9000, 1, seed=5)
    y = _gpu_mvm(_plan(fkt, X, kernel, ell, 5, 128, 0.5, alpha, scale), w)
    z = _oracle(orc, X, kernel, ell, 5, 128, 0.5, alpha, scale).mvm(w)
    assert _rel(y, z) < TOL


@pytest.mark.parametrize("kernel,ell", [("matern32", 0.2), ("gaussian", 0.1), ("laplace", 1.0), ("cauchy", 0.05)])
@pytest.mark.parametrize("d", [3, 4])
def test_near_four_targets_per_thread(fkt, orc, kernel, ell, d):
    """The register-blocked near-field variant (4 targets per thread) against the oracle."""
    X = inputs.gaussian_mixture(9000, d, 6, 0.07, seed=25)
    w = inputs.normal_weights(9000, 1, seed=26)
    plan = _plan(fkt, X, kernel, ell, 4, 128, 0.5)
    plan.set_option("near_targets_per_thread", "4")
    y = _gpu_mvm(plan, w)
    z = _oracle(orc, X, kernel, ell, 4, 128, 0.5).mvm(w)
    assert _rel(y, z) < TOL


@pytest.mark.parametrize("p", [0, 1, 2, 3, 6, 7, 8, 9, 10])
def test_orders_d3(fkt, orc, p):
    X = inputs.unit_ball(7000, 3, seed=6)
    w = inputs.normal_weights(7000, 1, seed=7)
    y = _gpu_mvm(_plan(fkt, X, "cauchy", 0.3, p, 96, 0.6), w)
    z = _oracle(orc, X, "cauchy", 0.3, p, 96, 0.6).mvm(w)
    assert _rel(y, z) < TOL


@pytest.mark.parametrize("nrhs", [2, 4, 8, 11, 20, 36, 53])
def test_multi_rhs(fkt, orc, nrhs):
    """Ragged right-hand-side groups and passes (8 per group, 32 per pass; 20 and 53 leave a
    32-wide near pass with fewer right-hand sides than its width; 2, 4 and the second pass of
    36 run the 4-wide near pass, whose records hold only 4 weights) against the oracle."""
    X = inputs.gaussian_mixture(12000, 3, 10, 0.05, seed=8)
    w = inputs.normal_weights(12000, nrhs, seed=9)
    y = _gpu_mvm(_plan(fkt, X, "matern32", 0.2, 6, 256, 0.5), w)
    z = _oracle(orc, X, "matern32", 0.2, 6, 256, 0.5).mvm(w)
    assert _rel(y, z) < TOL


@pytest.mark.parametrize("kernel,ell,p,nrhs", [("matern52", 0.3, 4, 1), ("matern52", 0.3, 6, 1),
                                                ("matern52", 0.3, 6, 8), ("ratquad", 0.3, 5, 3),
                                                ("gaussian", 0.2, 8, 1)])
def test_d4(fkt, orc, kernel, ell, p, nrhs):
    X = inputs.gaussian_mixture(8000, 4, 20, 0.05, seed=10)
    w = inputs.normal_weights(8000, nrhs, seed=11)
    y = _gpu_mvm(_plan(fkt, X, kernel, ell, p, 128, 0.5), w)
    z = _oracle(orc, X, kernel, ell, p, 128, 0.5).mvm(w)
    assert _rel(y, z) < TOL


# ------------------------------------------------------------- edge cases
def test_tiny_and_degenerate(fkt, orc):
    for X in (inputs.uniform_cube(1, 3), inputs.uniform_cube(2, 3), inputs.uniform_cube(37, 3),
              np.repeat(inputs.uniform_cube(1, 3), 300, axis=0)):
        w = inputs.normal_weights(len(X), 3, seed=12)
        for kernel in ("gaussian", "laplace"):
            plan = _plan(fkt, X, kernel, 0.5, 3, 16, 0.5)
            y = _gpu_mvm(plan, w)
            z = _oracle(orc, X, kernel, 0.5, 3, 16, 0.5).mvm(w)
            if np.linalg.norm(z) == 0:
                assert np.abs(y).max() == 0
            else:
                assert _rel(y, z) < TOL


def test_all_near_matches_dense(fkt, orc):
    """theta -> 0 (nothing far) and leaf_size >= N (one leaf): the FKT is the dense product."""
    X = inputs.uniform_cube(3000, 3, seed=13)
    w = inputs.normal_weights(3000, 2, seed=14)
    zd = orc.dense(X, orc.kparams("matern32", 0.2), w)
    for theta, leaf in ((1e-6, 64), (0.5, 4096)):
        plan = _plan(fkt, X, "matern32", 0.2, 4, leaf, theta)
        assert plan.stats()["far_pairs"] == 0
        assert _rel(_gpu_mvm(plan, w), zd) < TOL


def test_dense_gpu_matches_oracle(fkt, orc):
    import torch

    X = inputs.gaussian_mixture(5000, 3, 4, 0.1, seed=15)
    w = inputs.normal_weights(5000, 9, seed=16)
    plan = _plan(fkt, X, "cauchy", 0.05, 2, 64, 0.5)
    y = plan.dense(torch.from_numpy(w).cuda()).cpu().numpy()
    assert _rel(y, orc.dense(X, orc.kparams("cauchy", 0.05), w)) < TOL


def test_host_entry_matches_device_entry(fkt):
    import torch

    X = inputs.uniform_cube(9000, 3, seed=17)
    w = inputs.normal_weights(9000, 4, seed=18)
    plan = _plan(fkt, X, "gaussian", 0.1, 4, 256, 0.5)
    y_dev = plan.mvm(torch.from_numpy(w).cuda()).cpu().numpy()
    y_host = plan.mvm_host(w)
    np.testing.assert_array_equal(y_dev, y_host)


def test_repeatable(fkt):
    import torch

    X = inputs.uniform_cube(9000, 3, seed=19)
    w = torch.from_numpy(inputs.normal_weights(9000, 1, seed=20)).cuda()
    plan = _plan(fkt, X, "matern32", 0.2, 6, 256, 0.5)
    a = plan.mvm(w).cpu().numpy()
    b = plan.mvm(w).cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_invalid_device_arguments(fkt):
    import ctypes

    import torch

    X = torch.from_numpy(inputs.uniform_cube(100, 3)).cuda()
    h = ctypes.c_void_p()
    k = fkt.make_kernel("gaussian", 0.1)
    host = np.zeros((100, 3), np.float32)
    assert fkt.lib().fkt_plan(ctypes.c_void_p(host.ctypes.data), 100, 3, k, 4, 64, 0.5, None,
                              ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    bad = X.clone()
    bad[5, 1] = float("nan")
    assert fkt.lib().fkt_plan(ctypes.c_void_p(bad.data_ptr()), 100, 3, k, 4, 64, 0.5, None,
                              ctypes.byref(h)) == fkt.FKT_ERR_INVALID_ARG
    plan = _plan(fkt, X.cpu().numpy(), "gaussian", 0.1, 4, 64, 0.5)
    w = torch.zeros((65, 100), device="cuda")
    with pytest.raises(fkt.FktError):
        plan.mvm(w)


# ------------------------------------------------------------ full size
def test_full_size_matern_1m_sampled(fkt, orc):
    """N = 1,000,000 Gaussian-mixture points, Matern-3/2 l=0.2, p=6, leaf 512, theta 0.5 -- the benchmark
    launch -- checked on 300 sampled targets the oracle evaluates one by one."""
    import torch

    X = inputs.gaussian_mixture(1_000_000, 3, 10, 0.05)
    w = inputs.normal_weights(1_000_000)
    plan = _plan(fkt, X, "matern32", 0.2, 6, 512, 0.5)
    y = plan.mvm(torch.from_numpy(w).cuda()).cpu().numpy().astype(np.float64)
    idx = inputs.subsample(1_000_000, 300)
    z = _oracle(orc, X, "matern32", 0.2, 6, 512, 0.5).mvm(w, idx)
    assert_bars(y[:, idx], z, TOL, "matern32 1M float32 form")
