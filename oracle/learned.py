"""FP64 reference of the learned block-Jacobi correction (TEST INFRASTRUCTURE ONLY).

Only tests/ use this.  It restates, in plain numpy float64, the objects the library's learned
preconditioner computes on the GPU:

* the teacher T_b = A_by A_yy^{-1} A_yb with A = K + sigma2 I (block b, neighbours y), by a
  dense solve;
* the network V = Wo^T [phi(u_i); g; h] + bo with phi(u) = tanh(W2^T tanh(W1^T u + b1) + b2),
  g / h the means of phi over the block / the neighbours, u = (x - block centroid) / lengthscale;
* the loss L = sum_b |beta^2 V_b V_b^T - T_b|_F^2 / sum_b |T_b|_F^2 (beta fixed) and its gradient
  by reverse-mode differentiation written out by hand (pinned by finite differences in the tests).

Parameter vector layout: W1 [d][H], b1 [H], W2 [H][H], b2 [H], Wo [3H][R], bo [R], beta.
"""
from __future__ import annotations

import numpy as np


def shapes(d: int, H: int, R: int):
    sizes = [("W1", (d, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("Wo", (3 * H, R)), ("bo", (R,)),
             ("beta", (1,))]
    out, off = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = (off, shp)
        off += n
    return out, off


def unpack(params, d, H, R):
    lay, n = shapes(d, H, R)
    assert len(params) == n
    return {k: np.asarray(params[o:o + int(np.prod(s))], dtype=np.float64).reshape(s) for k, (o, s) in lay.items()}


def features(block_pts, nbr_pts, lengthscale):
    """u for the block points then the neighbours, relative to the block centroid."""
    block_pts = np.asarray(block_pts, np.float64)
    nbr_pts = np.asarray(nbr_pts, np.float64).reshape(-1, block_pts.shape[1])
    c = block_pts.mean(axis=0)
    return np.concatenate([block_pts, nbr_pts]) - c, len(block_pts)


def forward(p, U, n):
    A1 = U @ p["W1"] + p["b1"]
    Z1 = np.tanh(A1)
    A2 = Z1 @ p["W2"] + p["b2"]
    PHI = np.tanh(A2)
    g = PHI[:n].mean(axis=0)
    h = PHI[n:].mean(axis=0) if len(U) > n else np.zeros_like(g)
    F = np.concatenate([PHI[:n], np.tile(g, (n, 1)), np.tile(h, (n, 1))], axis=1)
    V = F @ p["Wo"] + p["bo"]
    return V, (U, Z1, PHI, g, h, F)


def loss_and_grad(params, d, H, R, blocks):
    """blocks: list of (U, n, D_b) with U from features(...) / lengthscale.  Returns (L, dL/dparams)."""
    p = unpack(params, d, H, R)
    beta2 = float(p["beta"][0]) ** 2
    normD = sum(float((D[:n, :n] ** 2).sum()) for _, n, D in blocks)
    grads = {k: np.zeros_like(v) for k, v in p.items()}
    L = 0.0
    for U, n, D in blocks:
        V, (U_, Z1, PHI, g, h, F) = forward(p, U, n)
        M = beta2 * V @ V.T - D[:n, :n]
        L += float((M ** 2).sum()) / normD
        dV = 4.0 * beta2 * (M @ V) / normD                 # M is symmetric
        grads["Wo"] += F.T @ dV
        grads["bo"] += dV.sum(axis=0)
        dF = dV @ p["Wo"].T                                # (n, 3H)
        dPHI = np.zeros_like(PHI)
        dPHI[:n] += dF[:, :H]
        dPHI[:n] += dF[:, H:2 * H].sum(axis=0) / n         # through g = mean over the block
        m = len(U) - n
        if m > 0:
            dPHI[n:] += dF[:, 2 * H:].sum(axis=0) / m      # through h = mean over the neighbours
        dA2 = dPHI * (1.0 - PHI ** 2)
        grads["W2"] += Z1.T @ dA2
        grads["b2"] += dA2.sum(axis=0)
        dZ1 = dA2 @ p["W2"].T
        dA1 = dZ1 * (1.0 - Z1 ** 2)
        grads["W1"] += U.T @ dA1
        grads["b1"] += dA1.sum(axis=0)
    lay, ntot = shapes(d, H, R)
    flat = np.zeros(ntot)
    for k, (o, s) in lay.items():
        if k != "beta":
            flat[o:o + int(np.prod(s))] = grads[k].ravel()
    return L, flat


def teacher(orc, kp, sigma2, block_pts, nbr_pts):
    """T_b = A_by A_yy^{-1} A_yb, A = K + sigma2 I, float64 dense solve (zero without neighbours)."""
    X = np.asarray(block_pts, np.float64)
    Y = np.asarray(nbr_pts, np.float64).reshape(-1, X.shape[1])
    if len(Y) == 0:
        return np.zeros((len(X), len(X)))
    Kfn = np.vectorize(lambda r: orc.kernel_value(kp, r))
    Ayy = Kfn(np.linalg.norm(Y[:, None] - Y[None], axis=2)) + sigma2 * np.eye(len(Y))
    Ayb = Kfn(np.linalg.norm(Y[:, None] - X[None], axis=2))
    return Ayb.T @ np.linalg.solve(Ayy, Ayb)
