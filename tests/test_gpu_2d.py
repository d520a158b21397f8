"""d = 2 (circular harmonics, Chebyshev zonal functions) on the GPU against the oracle.

The 2-D setting of the paper's Barnes-Hut comparison (Sec. 5.2): the Cauchy kernel on uniform
points in the unit square, orders p = 0 (one term per node, the Barnes-Hut monopole at the box
centre) up to 10, theta from 0.25 to 0.75.  Bars as elsewhere: trees and lists bit-identical,
the product within 1e-5 (relative 2-norm per right-hand side, and per target against the
largest |z|) of the oracle FKT, which itself matches the dense product within its truncation
error."""
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


@pytest.fixture(scope="module")
def square():
    X = inputs.uniform_cube(20000, 2, seed=11)
    W = inputs.normal_weights(20000, 8, seed=12)
    return X, W


def _plan(fkt, X, kernel, ell, p, leaf, theta):
    import torch

    return fkt.Plan(torch.from_numpy(X).cuda(), kernel, lengthscale=ell, p=p, leaf_size=leaf, theta=theta)


def test_tree_and_lists_identical_to_oracle_2d(fkt, orc, square):
    X, _ = square
    plan = _plan(fkt, X, "cauchy", 0.05, 4, 128, 0.5)
    ora = orc.FKT(X, orc.kparams("cauchy", 0.05), p=4, leaf_size=128, theta=0.5)
    g, o = plan.tree(), ora.tree()
    for k in ("perm", "begin", "end", "level", "leaf", "child"):
        np.testing.assert_array_equal(g[k], o[k], err_msg=k)
    np.testing.assert_array_equal(g["centre"], o["centre"])
    np.testing.assert_array_equal(g["rho2"], o["rho2"])
    far, near = plan.target_sets()
    rng = np.random.default_rng(1)
    for t in rng.choice(len(X), 300, replace=False):
        of, on = ora.target_lists(int(g["perm"][t]))
        assert sorted(far[t]) == sorted(of.tolist()), t
        assert sorted(near[t]) == sorted(on.tolist()), t


@pytest.mark.parametrize("theta", [0.25, 0.5, 0.75])
@pytest.mark.parametrize("p", [0, 2, 4, 6, 8, 10])
def test_cauchy_2d_matches_oracle(fkt, orc, square, p, theta):
    """Barnes-Hut (p = 0) through p = 10 at three acceptance parameters, 1 and 8 right-hand sides."""
    import torch

    X, W = square
    plan = _plan(fkt, X, "cauchy", 0.05, p, 128, theta)
    ora = orc.FKT(X, orc.kparams("cauchy", 0.05), p=p, leaf_size=128, theta=theta)
    rng = np.random.default_rng(p + int(100 * theta))
    idx = rng.choice(len(X), 300, replace=False)
    for nrhs in (1, 8):
        y = plan.mvm(torch.from_numpy(W[:nrhs]).cuda()).cpu().numpy().astype(np.float64)
        plan.check()
        z = ora.mvm(W[:nrhs], idx)
        assert_bars(y[:, idx], z, TOL, f"d=2 p={p} theta={theta} nrhs={nrhs}")
    plan.close()


def test_cauchy_2d_truncation_error_falls_with_p(fkt, orc, square):
    """Against the dense product the GPU is as accurate as the expansion itself, and the
    expansion's error falls as p grows (Barnes-Hut, p = 0, is the least accurate)."""
    import torch

    X, W = square
    idx = np.random.default_rng(4).choice(len(X), 400, replace=False)
    zd = orc.dense(X, orc.kparams("cauchy", 0.05), W[:1], idx)
    errs = []
    for p in (0, 2, 4, 8):
        plan = _plan(fkt, X, "cauchy", 0.05, p, 128, 0.5)
        y = plan.mvm(torch.from_numpy(W[:1]).cuda()).cpu().numpy().astype(np.float64)[:, idx]
        errs.append(np.linalg.norm(y - zd) / np.linalg.norm(zd))
        plan.close()
    assert errs[0] > errs[1] > errs[2] > errs[3], errs
    assert errs[3] < 1e-4, errs


@pytest.mark.parametrize("near", ["tf32x3", "f16x3"])
def test_2d_near_tensor_cores(fkt, orc, square, near):
    """32-wide passes: the near field on the tensor cores (the d = 3 kernels over the zero third
    coordinate), far field float32."""
    import torch

    X, _ = square
    W = inputs.normal_weights(len(X), 32, seed=13)
    plan = _plan(fkt, X, "cauchy", 0.05, 6, 128, 0.5)
    plan.set_option("near_precision", near)
    y = plan.mvm(torch.from_numpy(W).cuda()).cpu().numpy().astype(np.float64)
    plan.check()
    idx = np.random.default_rng(5).choice(len(X), 200, replace=False)
    z = orc.FKT(X, orc.kparams("cauchy", 0.05), p=6, leaf_size=128, theta=0.5).mvm(W, idx)
    assert_bars(y[:, idx], z, TOL, f"d=2 near {near}")


def test_2d_tensor_core_far_field_is_rejected(fkt, square):
    """The tensor-core far field is built for d = 3 and 4: a d = 2 plan asking for it fails
    loudly instead of computing something else."""
    import torch

    X, W = square
    plan = _plan(fkt, X, "cauchy", 0.05, 4, 128, 0.5)
    plan.set_option("far_precision", "bf16x3")
    with pytest.raises(fkt.FktError):
        plan.mvm(torch.from_numpy(W[:8]).cuda())
        plan.check()
