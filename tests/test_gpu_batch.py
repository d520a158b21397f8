"""Batching form: independent problems of uneven size and mixed kernels in one batched product
(one CUDA-graph launch), each problem checked against its own oracle FKT."""
import numpy as np
import pytest

from paper_2106_04487_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5
KERNELS = [("gaussian", 0.1, 1.0, 1.0), ("laplace", 1.0, 1.0, 1.0), ("ratquad", 0.2, 1.0, 1.0)]


@pytest.fixture(scope="module")
def fkt():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2106_04487_gb300 import build, fkt as F

    build.build()
    F.lib()
    return F


def _problems(count, lo, hi, seed):
    sizes = inputs.batch_sizes(count, lo, hi, seed=seed)
    return [(inputs.unit_ball(int(n), 3, seed=100 + i), *KERNELS[i % 3]) for i, n in enumerate(sizes)]


def _check_against_oracle(orc, probs, batch, W, Y, p, theta):
    for i, (X, kname, ell, alpha, scale) in enumerate(probs):
        lo, hi = batch.offsets[i], batch.offsets[i + 1]
        F = orc.FKT(X, orc.kparams(kname, ell, alpha=alpha, scale=scale), p=p, leaf_size=int(batch.leaf_sizes[i]),
                    theta=theta)
        z = F.mvm(W[:, lo:hi])
        err = max(np.linalg.norm(Y[r, lo:hi] - z[r]) / np.linalg.norm(z[r]) for r in range(len(W)))
        assert err < TOL, (i, kname, hi - lo, err)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_batch_matches_per_problem_oracle(fkt, orc, prec):
    import torch

    probs = _problems(12, 300, 20000, seed=3)
    batch = fkt.Batch(probs, p=4, leaf_size=128, theta=0.5)
    batch.set_option("far_precision", prec)
    W = inputs.normal_weights(batch.N, 8, seed=4)
    Wd = torch.from_numpy(W).cuda()
    Y1 = batch.mvm(Wd).cpu().numpy().astype(np.float64)
    Yd = torch.empty_like(Wd)
    batch.mvm(Wd, out=Yd)           # captured graph, first replay with new output buffer
    batch.mvm(Wd, out=Yd)           # graph replay
    batch.check()
    Y2 = Yd.cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(Y1, Y2)
    tol = TOL if prec == "fp32" else 3e-5
    for i, (X, kname, ell, alpha, scale) in enumerate(probs):
        lo, hi = batch.offsets[i], batch.offsets[i + 1]
        F = orc.FKT(X, orc.kparams(kname, ell, alpha=alpha, scale=scale), p=4, leaf_size=128, theta=0.5)
        z = F.mvm(W[:, lo:hi])
        err = max(np.linalg.norm(Y2[r, lo:hi] - z[r]) / np.linalg.norm(z[r]) for r in range(8))
        assert err < tol, (i, kname, hi - lo, err)
    assert batch.totals["nodes"] > 0 and batch.totals["near_pairs"] > 0


def test_batch_autotuned_leaf_sizes(fkt, orc):
    import torch

    probs = _problems(6, 2000, 40000, seed=5)
    batch = fkt.Batch(probs, p=4, leaf_size=0, theta=0.5)
    assert set(batch.leaf_sizes.tolist()) <= {64, 128, 256, 512}
    W = inputs.normal_weights(batch.N, 3, seed=6)
    Y = batch.mvm(torch.from_numpy(W).cuda()).cpu().numpy().astype(np.float64)
    _check_against_oracle(orc, probs, batch, W, Y, 4, 0.5)


def test_autotune_leaf_picks_a_candidate(fkt):
    import torch

    X = torch.from_numpy(inputs.uniform_cube(50000, 3, seed=7)).cuda()
    best, ms = fkt.fkt_autotune_leaf(X, fkt.make_kernel("gaussian", 0.1), 4, 0.5, nrhs=1, candidates=(128, 512))
    assert best in (128, 512) and ms > 0


def test_autotuned_batch_matches_oracle(fkt, orc):
    """Leaf sizes autotuned per size class (leaf_size = 0) and the kernel variants autotuned for 8
    and 32 right-hand sides (fkt_batch_autotune): whatever they pick, the product keeps the bars."""
    import torch

    sizes = inputs.batch_sizes(12, 2000, 40000, seed=91)
    kinds = [("gaussian", 0.1, 1.0, 1.0), ("laplace", 1.0, 1.0, 1.0), ("ratquad", 0.2, 1.0, 1.0)]
    probs = [(inputs.unit_ball(int(n), 3, seed=200 + i), *kinds[i % 3]) for i, n in enumerate(sizes)]
    batch = fkt.Batch(probs, p=4, leaf_size=0, theta=0.5)
    assert set(batch.leaf_sizes.tolist()) <= {64, 128, 256, 512}
    batch.set_option("far_precision", "bf16x3")
    for nrhs in (8, 32):
        chosen = batch.autotune(nrhs)
        assert "far_kernel=" in chosen and (nrhs <= 16 or "near_precision=" in chosen), chosen
        W = inputs.normal_weights(batch.N, nrhs, seed=92)
        Y = batch.mvm(torch.from_numpy(W).cuda()).cpu().numpy().astype(np.float64)
        batch.check()
        for i in (0, 1, 2, 11):
            X, kname, ell, alpha, scale = probs[i]
            lo, hi = batch.offsets[i], batch.offsets[i + 1]
            F = orc.FKT(X, orc.kparams(kname, ell, alpha=alpha, scale=scale), p=4,
                        leaf_size=int(batch.leaf_sizes[i]), theta=0.5)
            idx = inputs.subsample(hi - lo, 100, seed=93 + i)
            z = F.mvm(W[:, lo:hi], idx)
            err = max(np.linalg.norm(Y[r, lo + idx] - z[r]) / np.linalg.norm(z[r]) for r in range(nrhs))
            print(f"autotuned ({chosen}) nrhs={nrhs} problem {i} ({kname}): {err:.2e}")
            assert err < 3e-5, (nrhs, i, chosen, err)
