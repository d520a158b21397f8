"""Pins of the oracle's tree, interaction sets and whole FKT (Sec. 3.1-3.2, Algorithm 1)."""
import numpy as np
import pytest

from paper_2106_04487_gb300 import inputs


@pytest.fixture(scope="module")
def small(orc):
    X = inputs.gaussian_mixture(3000, 3, components=5, std=0.08)
    kp = orc.kparams("matern32", 0.2)
    F = orc.FKT(X, kp, p=4, leaf_size=64, theta=0.5)
    return X, kp, F


def test_tree_invariants(small):
    """Contract of Sec. 3.1 (midpoint splits cycling the axes): children partition the parent's range at a code bit,
    leaves hold <= leaf_size points, codes sorted, centres are box midpoints, rho2 is the max."""
    X, kp, F = small
    t = F.tree()
    N, d, B = len(X), 3, 21
    assert np.all(np.diff(t["codes"].astype(np.uint64)) >= 0)
    assert sorted(t["perm"]) == list(range(N))
    Xs = X[t["perm"]].astype(np.float64)
    leaf_pts = 0
    for i in range(len(t["begin"])):
        b, e, lev = t["begin"][i], t["end"][i], t["level"][i]
        assert e > b
        kids = [c for c in t["child"][i] if c >= 0]
        if t["leaf"][i]:
            assert not kids
            assert e - b <= 64 or lev == d * B
            leaf_pts += e - b
        else:
            assert e - b > 64
            assert t["begin"][kids[0]] == b and t["end"][kids[-1]] == e
            if len(kids) == 2:
                assert t["end"][kids[0]] == t["begin"][kids[1]]
            for c in kids:
                assert t["level"][c] == lev + 1
            # the split is at code bit `lev` from the top: that bit is 0 on the left, 1 on the right
            bit = np.uint64(d * B - 1 - lev)
            bits = (t["codes"][b:e] >> bit) & np.uint64(1)
            assert np.all(np.diff(bits.astype(np.int64)) >= 0)
        # every point of the node lies inside the node's box: |x - c|_inf <= half width (+ one quantum)
        c = t["centre"][i]
        for a in range(d):
            na = (lev - a + d - 1) // d if lev > a else 0
            half = t["L"] * 2.0 ** (-na - 1)
            assert np.all(np.abs(Xs[b:e, a] - c[a]) <= half + t["L"] * 2.0 ** -B)
        r2 = ((Xs[b:e] - c) ** 2).sum(1).max()
        assert t["rho2"][i] == pytest.approx(r2, rel=1e-14)
    assert leaf_pts == N


def test_coverage_invariant(small):
    """For every (target, source) exactly one of: source in a near leaf of the target, or
    source inside exactly one far node of the target; no far node has a far ancestor (Sec. 3.1:
    F_i disjoint along ancestor chains; N_l = points in no F_j on the path)."""
    X, kp, F = small
    t = F.tree()
    inv = np.empty(len(X), np.int64)
    inv[t["perm"]] = np.arange(len(X))
    rng = np.random.default_rng(0)
    theta2 = 0.25
    for tgt in rng.choice(len(X), 200, replace=False):
        far, near = F.target_lists(tgt)
        cover = np.zeros(len(X), np.int64)
        x = X[tgt].astype(np.float64)
        for b in far:
            cover[t["begin"][b]:t["end"][b]] += 1
            d2 = ((x - t["centre"][b]) ** 2).sum()
            assert t["rho2"][b] < theta2 * d2
        for b in near:
            assert t["leaf"][b]
            cover[t["begin"][b]:t["end"][b]] += 1
        assert np.all(cover == 1)
        assert inv[tgt] in np.concatenate([np.arange(t["begin"][b], t["end"][b]) for b in near])


def test_all_near_equals_dense(orc):
    """theta -> 0: nothing is far, so the FKT is the dense MVM (eq. nbody) up to rounding order."""
    X = inputs.uniform_cube(1500, 3, seed=4)
    w = inputs.normal_weights(1500, 2)
    for kname, ell in (("gaussian", 0.1), ("laplace", 1.0)):
        kp = orc.kparams(kname, ell)
        F = orc.FKT(X, kp, p=2, leaf_size=32, theta=1e-9)
        np.testing.assert_allclose(F.mvm(w), orc.dense(X, kp, w), rtol=1e-12, atol=1e-10)
        F = orc.FKT(X, kp, p=2, leaf_size=5000, theta=0.5)   # one leaf holding everything
        np.testing.assert_allclose(F.mvm(w), orc.dense(X, kp, w), rtol=1e-12, atol=1e-10)


def test_fkt_error_decays_with_p(orc):
    """Whole-FKT error against dense decreases with p at fixed tree and theta (Sec. 4.1)."""
    X = inputs.uniform_cube(4000, 3, seed=2)
    w = inputs.normal_weights(4000)
    kp = orc.kparams("matern32", 0.2)
    zd = orc.dense(X, kp, w)
    errs = []
    for p in (0, 2, 4, 6, 8):
        z = orc.FKT(X, kp, p=p, leaf_size=64, theta=0.5).mvm(w)
        errs.append(np.linalg.norm(z - zd) / np.linalg.norm(zd))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4


def test_dense_kernel_matrix_symmetric(orc):
    """K_ij = K(|r_i - r_j|) is symmetric: u^T (K v) = v^T (K u)."""
    X = inputs.unit_ball(800, 3, seed=6)
    u = inputs.normal_weights(800, seed=7)[0]
    v = inputs.normal_weights(800, seed=8)[0]
    kp = orc.kparams("cauchy", 0.3)
    assert u @ orc.dense(X, kp, v)[0] == pytest.approx(v @ orc.dense(X, kp, u)[0], rel=1e-12)


def test_dense_subsample_matches_full(orc):
    X = inputs.uniform_cube(1000, 3, seed=5)
    w = inputs.normal_weights(1000, 3)
    kp = orc.kparams("gaussian", 0.2)
    full = orc.dense(X, kp, w)
    idx = inputs.subsample(1000, 50)
    np.testing.assert_array_equal(orc.dense(X, kp, w, idx), full[:, idx])


def test_fkt_subsample_matches_full(orc, small):
    X, kp, F = small
    w = inputs.normal_weights(len(X), 2)
    full = F.mvm(w)
    idx = inputs.subsample(len(X), 40)
    np.testing.assert_allclose(F.mvm(w, idx), full[:, idx], rtol=1e-14, atol=1e-14)


def test_duplicate_points_and_max_depth(orc):
    """Exact duplicates cannot be separated: the leaf at level d*B may exceed leaf_size;
    the singular kernel skips r = 0 pairs."""
    X = np.repeat(inputs.uniform_cube(30, 3, seed=9), 20, axis=0)
    w = inputs.normal_weights(len(X))
    for kname in ("laplace", "cauchy"):
        kp = orc.kparams(kname, 0.5)
        F = orc.FKT(X, kp, p=3, leaf_size=8, theta=0.5)
        t = F.tree()
        assert (t["end"] - t["begin"])[t["leaf"]].max() == 20
        assert t["level"].max() == 63
        z, zd = F.mvm(w), orc.dense(X, kp, w)
        # identical points get identical results
        assert np.all(z.reshape(30, 20) == z.reshape(30, 20)[:, :1])
        near_only = orc.FKT(X, kp, p=3, leaf_size=8, theta=1e-9).mvm(w)
        np.testing.assert_allclose(near_only, zd, rtol=1e-12, atol=1e-10)
        z8 = orc.FKT(X, kp, p=8, leaf_size=8, theta=0.5).mvm(w)
        assert np.linalg.norm(z8 - zd) < np.linalg.norm(z - zd)
