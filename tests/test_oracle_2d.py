"""Pins of the oracle's d = 2 expansion (alpha = 0, Chebyshev zonal functions) against what the
mathematics fixes independently of the oracle: numpy's Chebyshev change of basis, the 2-D
addition theorem, the modified-Bessel (Jacobi-Anger) expansion of the Gaussian, convergence in
p, and the all-near limit of the FKT."""
import numpy as np
import pytest

from oracle import oracle as orc_mod
from oracle import tables
from paper_2106_04487_gb300 import inputs


@pytest.fixture(scope="module")
def orc():
    orc_mod.build()
    return orc_mod


@pytest.mark.parametrize("i", range(12))
def test_chebyshev_change_of_basis(i):
    """cos^i = sum_k A_{k,i} T_k (the d = 2 reading of eq. coschange) against numpy's
    monomial-to-Chebyshev conversion."""
    from numpy.polynomial import chebyshev

    want = chebyshev.poly2cheb([0.0] * i + [1.0])
    got = [float(tables.A(k, i, 2)) for k in range(i + 1)]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def test_harmonic_dims_2d():
    assert [tables.harmonic_dim(k, 2) for k in range(6)] == [1, 2, 2, 2, 2, 2]
    assert tables.num_terms(6, 2) == sum((1 if k == 0 else 2) * ((6 - k) // 2 + 1) for k in range(7))


def test_addition_theorem_2d(orc):
    """sum_h Y_kh(u) Y_kh(v) = T_k(u . v) = cos(k (phi_u - phi_v)) for the oracle's basis."""
    b = orc.Basis(2, 8)
    rng = np.random.default_rng(3)
    for _ in range(20):
        pu, pv = rng.uniform(0, 2 * np.pi, 2)
        u, v = np.array([np.cos(pu), np.sin(pu)]), np.array([np.cos(pv), np.sin(pv)])
        Yu, Yv = b.harmonics(u), b.harmonics(v)
        off = 0
        for k in range(9):
            D = tables.harmonic_dim(k, 2)
            s = float(Yu[off:off + D] @ Yv[off:off + D])
            assert abs(s - np.cos(k * (pu - pv))) < 1e-12, (k, s)
            off += D


@pytest.mark.parametrize("ell", [0.7, 1.0, 1.6])
def test_gaussian_degree_k_is_modified_bessel(orc, ell):
    """exp(-|x - x'|^2 / (2 l^2)) = exp(-(r^2 + r'^2) / (2 l^2)) [I_0(z) + 2 sum_k I_k(z) T_k(cos g)],
    z = r r' / l^2 (generating function of the modified Bessel functions).  The degree-k radial
    function of the expansion (eq. kdef with the d = 2 table) must equal its k-th term."""
    from scipy.special import iv

    kp = orc.kparams("gaussian", ell)
    P = 30
    for r, rp in [(1.5, 0.5), (2.0, 0.3), (1.0, 0.45)]:
        Kd = orc.kernel_derivs(kp, r, P)          # K^(m)(r), m = 0..P (the oracle's jets)
        z = r * rp / ell ** 2
        pref = np.exp(-(r * r + rp * rp) / (2 * ell * ell))
        for k in range(11):
            g = 0.0
            for j in range(k, P + 1, 2):
                g += rp ** j * sum(Kd[m] * r ** (m - j) * float(tables.Tbar(k, j, m, 2)) for m in range(j + 1))
            want = pref * (1.0 if k == 0 else 2.0) * iv(k, z)
            assert abs(g - want) <= 1e-12 + 1e-9 * abs(want), (r, rp, k, g, want)


@pytest.mark.parametrize("kernel,ell", [("cauchy", 1.0), ("matern32", 1.0), ("exponential", 2.0), ("laplace", 1.0)])
def test_expansion_converges_in_p_2d(orc, kernel, ell):
    """Error of the truncated expansion against the kernel itself decays with p at |x'|/|x| = 1/3."""
    rng = np.random.default_rng(5)
    kp = orc.kparams(kernel, ell)
    n = 300
    ang = rng.uniform(0, 2 * np.pi, (n, 2))
    X = 1.5 * np.stack([np.cos(ang[:, 0]), np.sin(ang[:, 0])], axis=1)
    XP = 0.5 * np.stack([np.cos(ang[:, 1]), np.sin(ang[:, 1])], axis=1)
    direct = np.array([orc.kernel_value(kp, float(np.linalg.norm(a - b))) for a, b in zip(X, XP)])
    errs = [np.abs(orc.expansion_gegenbauer(2, p, kp, X, XP) - direct).max() for p in (2, 6, 12, 24)]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[3] < 1e-6 * np.abs(direct).max(), errs
    # the harmonic basis gives the same truncated expansion as the zonal (Chebyshev) form
    b = orc.Basis(2, 12)
    np.testing.assert_allclose(b.expansion(kp, X, XP), orc.expansion_gegenbauer(2, 12, kp, X, XP), rtol=1e-11,
                               atol=1e-13)


def test_fkt_2d_all_near_equals_dense(orc):
    """theta -> 0 makes every node near: the FKT is then the dense product (Algorithm 1)."""
    X = inputs.uniform_cube(600, 2, seed=7)
    W = inputs.normal_weights(600, 2, seed=8)
    kp = orc.kparams("cauchy", 0.05)
    z = orc.FKT(X, kp, p=4, leaf_size=32, theta=1e-6).mvm(W)
    np.testing.assert_allclose(z, orc.dense(X, kp, W), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("p,bar", [(4, 2e-3), (8, 1e-4)])
def test_fkt_2d_cauchy_within_truncation(orc, p, bar):
    """The 2-D Cauchy product on uniform points in the unit square (Sec. 5.2's setting, smaller N)
    matches the dense product within the truncation error, which falls with p."""
    X = inputs.uniform_cube(3000, 2, seed=9)
    W = inputs.normal_weights(3000, 1, seed=10)
    kp = orc.kparams("cauchy", 0.05)
    z = orc.FKT(X, kp, p=p, leaf_size=64, theta=0.5).mvm(W)
    y = orc.dense(X, kp, W)
    err = np.linalg.norm(z - y) / np.linalg.norm(y)
    assert err < bar, err
