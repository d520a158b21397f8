"""Learned low-rank correction of the block-Jacobi preconditioner (GPU) against the float64
reference: the teacher blocks T_b = A_by A_yy^-1 A_yb, the loss and its gradient at the same
parameters, the effect of training, and the corrected preconditioner inside fkt_solve (with its
block-Jacobi fallback)."""
import numpy as np
import pytest

from oracle import learned
from paper_2106_04487_gb300 import inputs

pytestmark = pytest.mark.gpu

SIGMA2, ELL = 1e-2, 0.3


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
def trained(fkt):
    import torch

    X = inputs.gaussian_mixture(20000, 4, 20, 0.05, seed=50)
    plan = fkt.Plan(torch.from_numpy(X).cuda(), "matern52", lengthscale=ELL, p=6, leaf_size=256, theta=0.3)
    info = plan.learn_precond(SIGMA2, rank=8, hidden=32, steps=300, lr=3e-3, train_blocks=64, seed=1)
    return X, plan, info


def _block_data(X, plan, b):
    perm = plan.tree()["perm"]
    rng = plan.lists()["block_range"]
    Xs = X[perm].astype(np.float64)
    lo, hi = rng[b]
    nbr = []
    if b > 0:
        plo, phi = rng[b - 1]
        nbr.append(Xs[max(plo, phi - 32):phi])
    if b + 1 < len(rng):
        nlo, nhi = rng[b + 1]
        nbr.append(Xs[nlo:min(nhi, nlo + 32)])
    nbr = np.concatenate(nbr) if nbr else np.zeros((0, X.shape[1]))
    return Xs[lo:hi], nbr


def test_teacher_blocks_match_float64(fkt, orc, trained):
    X, plan, info = trained
    blocks, T = plan.learn_teacher(info["ntrain"])
    kp = orc.kparams("matern52", ELL)
    for k in (0, 7, info["ntrain"] - 1):
        xb, nb = _block_data(X, plan, int(blocks[k]))
        ref = learned.teacher(orc, kp, SIGMA2, xb, nb)
        n = len(xb)
        got = T[k][:n, :n].astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-2, k


def test_gpu_loss_and_gradient_match_float64(fkt, trained):
    """Forward and backward kernels against the float64 reference, on the GPU's own teacher data."""
    X, plan, info = trained
    blocks, D = plan.learn_teacher(info["ntrain"])
    data = []
    for k, b in enumerate(blocks):
        xb, nb = _block_data(X, plan, int(b))
        U, n = learned.features(xb, nb, ELL)
        data.append((U / ELL, n, D[k].astype(np.float64)))
    params = plan.learn_params()
    for prm in (params, params + 0.01 * np.random.default_rng(0).standard_normal(len(params)).astype(np.float32)):
        prm = prm.astype(np.float32)
        prm[-1] = params[-1]
        loss_gpu, grad_gpu = plan.learn_eval(prm)
        loss_ref, grad_ref = learned.loss_and_grad(prm.astype(np.float64), 4, 32, 8, data)
        assert abs(loss_gpu - loss_ref) < 1e-3 * abs(loss_ref), (loss_gpu, loss_ref)
        assert np.linalg.norm(grad_gpu - grad_ref) < 2e-3 * np.linalg.norm(grad_ref)


def test_training_reduces_the_objective(trained):
    """What the trained network gains over no correction: most of the teacher is reproduced."""
    X, plan, info = trained
    print(info)
    assert info["loss_initial"] > 0.5
    assert info["loss_final"] < 0.1 * info["loss_initial"], info


def test_solve_with_learned_correction(fkt, trained):
    """The corrected preconditioner inside CG converges to the requested residual with the true
    residual as the judge (falling back to block-Jacobi if it does not); the iteration counts of the
    three preconditioners are printed.  No iteration gain is asserted because none was measured: for
    this long-range kernel no block-diagonal preconditioner beats none -- CG's slow directions are
    smooth modes spanning many blocks, which a block-local correction cannot represent -- and the
    learned blocks take about as many iterations as block-Jacobi (measured at N = 20k, d = 4,
    tol 1e-5: none 2105, block-Jacobi 3675, learned 4015-4210).  What the network does gain is
    asserted in test_training_reduces_the_objective."""
    import torch

    X, plan, info = trained
    b = torch.from_numpy(inputs.normal_weights(len(X), 2, seed=51)).cuda()
    its = {}
    for pc in ("none", "block_jacobi", "learned"):
        plan.set_option("preconditioner", pc)
        x, st = plan.solve(SIGMA2, b, tol=1e-5, max_iter=6000, raise_on_not_converged=False)
        its[pc] = (st["iterations"], st["converged"], st["used_fallback"], st["true_rel_residual"])
    print(its)
    assert its["learned"][1] == 1
    assert its["learned"][3] < 5e-3
