"""Tests of the analysis layer (paper_2304_03311_gb300/analysis.py), CPU only.

Each function is pinned to something other than itself: closed forms of the
theta and eta functions at tau = i, an independent mpmath evaluation of the
RVB and AdS shapes from their printed definitions (the library removes the
endpoint singularities by substitution, mpmath integrates the originals),
Appendix C's expansion checked against actual finite differences, recovery
of known parameters by the fits, and the exact transfer-matrix c-function.
"""
import math

import numpy as np
import pytest

import oracle.estimator as oest
import oracle.exact as ex
from paper_2304_03311_gb300 import analysis as an

mp = pytest.importorskip("mpmath")


def test_c_function_matches_the_oracle_and_symmetry():
    for d, L in ((2, 64), (3, 16)):
        for l in (0, 3, L // 2 - 1):
            assert an.c_function(0.37, d, L, l) == pytest.approx(
                oest.c_function(0.37, d, L, l), rel=1e-14)
    c, e = an.c_function([0.1, 0.2], 2, 10, [1, 8], err=[0.01, 0.02])
    assert e[0] / c[0] == pytest.approx(0.1)


def test_increments_sum_to_the_entropy():
    ds = np.array([0.3, 0.1, 0.05])
    s, e = an.renyi_from_increments(ds, [0.01, 0.02, 0.02])
    np.testing.assert_allclose(s, [0, 0.3, 0.4, 0.45])
    assert e[-1] == pytest.approx(0.03)


def test_theta_and_eta_closed_forms_at_tau_i():
    # theta_3(i) = pi^(1/4)/Gamma(3/4); eta(i) = Gamma(1/4)/(2 pi^(3/4))
    assert an.theta3_imag(1.0) == pytest.approx(math.pi ** 0.25 / math.gamma(0.75), rel=1e-14)
    assert an.eta_imag(1.0) == pytest.approx(math.gamma(0.25) / (2 * math.pi ** 0.75),
                                             rel=1e-14)
    for t in (0.07, 0.3, 0.9, 1.7, 4.0):
        q = mp.exp(-mp.pi * t)
        assert an.theta3_imag(t) == pytest.approx(float(mp.jtheta(3, 0, q)), rel=1e-13)
        eta = mp.exp(-mp.pi * t / 12) * mp.nprod(lambda n: 1 - mp.exp(-2 * mp.pi * n * t),
                                                 [1, mp.inf])
        assert an.eta_imag(t) == pytest.approx(float(eta), rel=1e-12)


def _rvb_mpmath(x, t=1.0):
    th = lambda s: mp.jtheta(3, 0, mp.exp(-mp.pi * s))
    eta = lambda s: mp.exp(-mp.pi * s / 12) * mp.nprod(
        lambda n: 1 - mp.exp(-2 * mp.pi * n * s), [1, mp.inf])
    v = eta(t) ** 2 / (th(2 * t) * th(t / 2)) * th(2 * x * t) * th(2 * (1 - x) * t) / (
        eta(2 * x * t) * eta(2 * (1 - x) * t))
    return float(-2 * mp.log(v))


@pytest.mark.parametrize("x", [0.05, 0.2, 0.5])
def test_rvb_shape_against_mpmath(x):
    assert an.g_rvb(x) == pytest.approx(_rvb_mpmath(x), rel=1e-11, abs=1e-12)
    assert an.g_rvb(1 - x) == pytest.approx(an.g_rvb(x), rel=1e-12)


def _ads_mpmath(chi):
    P = lambda y: 1 - chi * y ** 3 - (1 - chi) * y ** 4
    xi = mp.quad(lambda y: y ** 2 / ((1 - chi * y ** 3) * mp.sqrt(P(y))), [0, 1])
    x = 3 / (2 * mp.pi) * mp.cbrt(chi) * mp.sqrt(1 - chi) * xi
    gi = mp.quad(lambda y: (1 / mp.sqrt(P(y)) - 1) / y ** 2, [0, 1])
    return float(x), float(chi ** (-mp.mpf(1) / 3) * (gi - 1))


@pytest.mark.parametrize("chi", [0.001, 0.2, 0.7, 0.97])
def test_ads_shape_against_mpmath(chi):
    mp.mp.dps = 30
    x, g = _ads_mpmath(mp.mpf(chi))
    assert an.ads_x_of_chi(chi) == pytest.approx(x, rel=1e-11)
    assert an.g_ads(x) == pytest.approx(g, rel=1e-9)
    assert an.g_ads(1 - x) == pytest.approx(g, rel=1e-9)


def test_small_x_limits_of_the_3d_c_functions():
    # RVB and AdS: dg/dx ~ x^-2, so C tends to a non-zero constant; 2D: C -> 0
    xs = np.array([1e-3, 2e-3, 4e-3])
    for fam in ("rvb", "ads"):
        c = an.c_function_family(fam, xs)
        assert np.all(c > 0.05)
        assert np.ptp(c) < 0.01 * c[0]
    c2 = an.c_function_family("2d", xs)
    np.testing.assert_allclose(c2 / xs, 0.5, rtol=5e-4)
    # the closed form of the 2D family = the generic definition
    gen = np.sin(math.pi * xs) ** 2 / (2 * math.pi ** 2) * an._derivative(an.g_2d, xs)
    np.testing.assert_allclose(an.c_function_family("2d", xs), gen, rtol=1e-7)


def test_fit_2d_recovers_k_and_has_unit_pulls():
    L, k = 64, 0.14
    l = np.arange(L - 1)
    x = an.midpoint_x(l, L)
    truth = an.fit_function_2d(x, k, L)
    err = np.full_like(x, 2e-3)
    rng = np.random.default_rng(0)
    pulls, chi2 = [], []
    for _ in range(200):
        f = an.fit_2d(x, truth + err * rng.standard_normal(len(x)), err, L)
        pulls.append((f.params[0] - k) / f.errors[0])
        chi2.append(f.chi2_per_dof)
    assert abs(np.mean(pulls)) < 0.25 and 0.8 < np.std(pulls) < 1.2
    assert 0.9 < np.mean(chi2) < 1.1
    exact = an.fit_2d(x, truth, err, L)
    assert exact.params[0] == pytest.approx(k, rel=1e-10)
    assert an.chi2_scaling_function_2d(x, an.scaling_function_2d(x), err).chi2 == 0.0


def test_fit_2d_on_the_exact_c_function():
    """At L_t = 8L the exact c-function of the transfer matrix gives k in the
    range of the paper's fits (0.138 to 0.162 at L = 32 ... 128)."""
    L = 12
    ds = ex.delta_s2_transfer(2, L, 8 * L, an.BETA_C_2D)
    l = np.arange(L)
    c = an.c_function(ds, 2, L, l)
    f = an.fit_2d(an.midpoint_x(l, L), c, np.full(L, 1e-3), L, drop_ends=1)
    assert 0.12 < f.params[0] < 0.22


@pytest.mark.parametrize("family", ["2d", "rvb", "ads"])
def test_family_fits_recover_parameters(family):
    x = an.midpoint_x(np.arange(1, 23), 24)
    s = an.FAMILIES[family](x, 0.11, 0.35)
    fs = an.fit_entropy(family, x, s, np.full_like(x, 1e-3))
    np.testing.assert_allclose(fs.params, [0.11, 0.35], rtol=1e-9)
    cf = an.c_function_family(family, x, 0.11)
    fc = an.fit_c_function(family, x, cf, np.full_like(x, 1e-3))
    assert fc.params[0] == pytest.approx(0.11, rel=1e-9)


def test_finite_difference_systematic_matches_actual_differences():
    """For S(x) = g_2D, the actual finite-difference c-function minus the exact
    one equals Appendix C's term up to O(1/L^4)."""
    d, c = 3, 0.2
    g = lambda x: an.g_2d(x, c)
    for L in (24, 48):
        l = np.arange(2, L // 2)
        x = an.midpoint_x(l, L)
        ds = g((l + 1) / L) - g(l / L)
        c_mc = an.c_function(ds, d, L, l)
        c_exact = an.c_function_family("2d", x, c)
        third = 2 * c * math.pi ** 3 / np.tan(math.pi * x) / np.sin(math.pi * x) ** 2
        np.testing.assert_allclose(an.third_derivative(g, x), third, rtol=3e-3)
        sys_term = an.finite_difference_systematic(d, L, x, third)
        resid = (c_mc - c_exact) - sys_term
        assert np.max(np.abs(resid)) < 0.05 * np.max(np.abs(sys_term))


def test_kramers_wannier_dual():
    assert an.kramers_wannier_dual(an.BETA_C_2D) == pytest.approx(an.BETA_C_2D, rel=1e-13)
    b = np.linspace(0.1, 1.0, 10)
    np.testing.assert_allclose(an.kramers_wannier_dual(an.kramers_wannier_dual(b)), b,
                               rtol=1e-12)
    assert np.all(np.diff(an.kramers_wannier_dual(b)) < 0)
