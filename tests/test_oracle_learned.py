"""Pins of the float64 reference of the learned preconditioner correction (no GPU)."""
import numpy as np

from oracle import learned


def _random_case(seed=0, d=3, H=8, R=3, nblocks=3):
    rng = np.random.default_rng(seed)
    lay, n = learned.shapes(d, H, R)
    params = 0.5 * rng.standard_normal(n)
    params[-1] = 0.7  # beta
    blocks = []
    for b in range(nblocks):
        nb, m = 5 + b, (0 if b == 0 else 4)
        U = rng.standard_normal((nb + m, d))
        Q = rng.standard_normal((nb, nb))
        D = Q @ Q.T / nb
        blocks.append((U, nb, D))
    return params, blocks, (d, H, R)


def test_gradient_matches_finite_differences():
    params, blocks, (d, H, R) = _random_case()
    L, g = learned.loss_and_grad(params, d, H, R, blocks)
    eps = 1e-6
    rng = np.random.default_rng(1)
    for i in rng.choice(len(params) - 1, 40, replace=False):
        e = np.zeros_like(params)
        e[i] = eps
        fd = (learned.loss_and_grad(params + e, d, H, R, blocks)[0] - learned.loss_and_grad(params - e, d, H, R, blocks)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert g[-1] == 0.0  # beta is not trained


def test_loss_is_zero_at_exact_fit_and_normalised():
    """With D_b = beta^2 V V^T for the network's own V, the loss vanishes; with V = 0 it is 1."""
    params, blocks, (d, H, R) = _random_case(seed=2)
    p = learned.unpack(params, d, H, R)
    exact = [(U, n, float(p["beta"][0]) ** 2 * learned.forward(p, U, n)[0] @ learned.forward(p, U, n)[0].T)
             for U, n, _ in blocks]
    assert learned.loss_and_grad(params, d, H, R, exact)[0] < 1e-24
    zero = params.copy()
    lay, _ = learned.shapes(d, H, R)
    o, s = lay["Wo"]
    zero[o:o + int(np.prod(s))] = 0.0
    o, s = lay["bo"]
    zero[o:o + int(np.prod(s))] = 0.0
    assert abs(learned.loss_and_grad(zero, d, H, R, blocks)[0] - 1.0) < 1e-12


def test_teacher_is_the_psd_coupling_term(orc):
    """T_b = A_by A_yy^-1 A_yb is what the Schur complement subtracts: A_bb - T_b = S, T_b >= 0,
    and T_b = 0 without neighbours."""
    rng = np.random.default_rng(3)
    X = rng.random((12, 3))
    Y = rng.random((7, 3))
    kp = orc.kparams("matern52", 0.3)
    T = learned.teacher(orc, kp, 1e-2, X, Y)
    P = np.concatenate([X, Y])
    Kfn = np.vectorize(lambda r: orc.kernel_value(kp, r))
    A = Kfn(np.linalg.norm(P[:, None] - P[None], axis=2)) + 1e-2 * np.eye(19)
    S_inv = np.linalg.inv(A)[:12, :12]              # inverse of the Schur complement
    np.testing.assert_allclose(A[:12, :12] - T, np.linalg.inv(S_inv), rtol=1e-7, atol=1e-9)
    assert np.linalg.eigvalsh((T + T.T) / 2).min() > -1e-10
    assert np.all(learned.teacher(orc, kp, 1e-2, X, np.zeros((0, 3))) == 0)
