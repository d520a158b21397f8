"""Host-side checks of the random Fourier frequencies behind fkt_solve's coarse space.

fkt_spectral_sample draws omega from each kernel's spectral density; by Bochner's theorem the
average of cos(omega . delta) over the draws must approach K(|delta|) / K(0).  The kernel values
come from the float64 oracle's closed forms, so a wrong density (a wrong number of degrees of
freedom, a missing factor in the scale) fails here.  No GPU is needed: the call does host work only.
"""
import numpy as np
import pytest

from paper_2106_04487_gb300 import fkt

R = 200_000
TOL = 8e-3   # 5 standard deviations of a mean of R values of cos, |cos| <= 1


@pytest.fixture(scope="module")
def F():
    from paper_2106_04487_gb300 import build

    build.build()
    fkt.lib()
    return fkt


@pytest.mark.parametrize("d", [3, 4])
@pytest.mark.parametrize("name,ell,alpha", [("gaussian", 0.3, 1.0), ("exponential", 0.3, 1.0), ("matern32", 0.3, 1.0),
                                            ("matern52", 0.3, 1.0), ("cauchy", 0.3, 1.0), ("ratquad", 0.3, 0.7),
                                            ("matern52", 0.05, 1.0)])
def test_frequencies_reproduce_the_kernel(F, orc, d, name, ell, alpha):
    omega, phase = F.fkt_spectral_sample(F.make_kernel(name, ell, alpha=alpha), d, R, seed=7)
    kp = orc.kparams(name, ell, alpha=alpha)
    k0 = orc.kernel_value(kp, 0.0)
    u = np.random.default_rng(d).standard_normal(d)
    u /= np.linalg.norm(u)
    for r in (0.15 * ell, 0.5 * ell, ell, 2 * ell):
        mc = np.cos(omega @ (r * u)).mean()
        want = orc.kernel_value(kp, r) / k0
        assert abs(mc - want) < TOL, (name, d, r, mc, want)
    assert phase.min() >= 0.0 and phase.max() < 2 * np.pi
    assert abs(np.cos(phase).mean()) < TOL


def test_sampler_is_seeded_and_validates(F):
    k = F.make_kernel("matern52", 0.3)
    a = F.fkt_spectral_sample(k, 4, 64, seed=3)
    b = F.fkt_spectral_sample(k, 4, 64, seed=3)
    c = F.fkt_spectral_sample(k, 4, 64, seed=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    L = F.lib()
    buf = np.zeros(64)
    for d, r, kern in ((0, 4, k), (9, 4, k), (3, 0, k), (3, 4, F.make_kernel("gaussian", -1.0)),
                       (3, 4, F.make_kernel("ratquad", 0.3, alpha=0.0))):
        assert L.fkt_spectral_sample(kern, d, r, 1, F._ptr(buf), F._ptr(buf)) == F.FKT_ERR_INVALID_ARG
    assert L.fkt_spectral_sample(k, 3, 4, 1, None, F._ptr(buf)) == F.FKT_ERR_INVALID_ARG
