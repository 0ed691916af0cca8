"""Pins of the oracle's FP64 estimator.

* ln <e^-W> against 60-digit arithmetic (mpmath), including works far outside
  the range where a naive exp would under/overflow.
* Closed forms: a constant work W gives ln <e^-W> = -W; forward and reverse
  signs of Delta S_2 (Appendix A, eq. equality_of_direct_reverse_protocols).
* The blocked jackknife of a plain mean equals the standard error of the block
  means (an exact identity for equal blocks).
* The symmetrised c-function (section 2) applied to the cylinder CFT increments
  reproduces C_2(x) = cos(pi x)/16 (section 2, c = 1/2, n = 2) as L grows.
"""
import math

import mpmath
import numpy as np
import pytest

import oracle.estimator as est


def _lme_mp(w):
    mpmath.mp.dps = 60
    s = mpmath.fsum(mpmath.exp(-mpmath.mpf(float(x))) for x in w)
    return float(mpmath.log(s / len(w)))


@pytest.mark.parametrize("scale,shift", [(1.0, 0.0), (30.0, 0.0), (5.0, 800.0), (5.0, -800.0)])
def test_log_mean_exp_matches_high_precision(scale, shift):
    rng = np.random.default_rng(int(scale * 7 + abs(shift) + (shift < 0)))
    w = rng.normal(shift, scale, size=2000)
    got = est.log_mean_exp_neg(w)
    ref = _lme_mp(w)
    assert abs(got - ref) <= 1e-13 * max(1.0, abs(ref))


def test_log_mean_exp_constant_and_single():
    assert est.log_mean_exp_neg(np.full(17, 3.25)) == pytest.approx(-3.25, abs=1e-15)
    assert est.log_mean_exp_neg([-2.0]) == 2.0
    with pytest.raises(ValueError):
        est.log_mean_exp_neg([])


def test_work_scaling_and_direction_signs():
    wi = np.array([4, -2, 0, 6, 2], dtype=np.int64)
    beta, N = 0.3, 7
    w = beta * wi / N
    ref = -_lme_mp(w)
    assert est.delta_s2(wi, beta, N, 1) == pytest.approx(ref, rel=1e-14)
    assert est.delta_s2(wi, beta, N, -1) == pytest.approx(-ref, rel=1e-14)
    assert est.delta_s2(wi, 0.0, N, 1) == 0.0


def test_jackknife_blocks_layout():
    assert est.jackknife_blocks(100, 32) == [(i * 3, i * 3 + 3) for i in range(31)] + [(93, 100)]
    assert est.jackknife_blocks(5, 32) == [(i, i + 1) for i in range(5)]


def test_jackknife_of_mean_is_standard_error_of_block_means():
    rng = np.random.default_rng(1)
    x = rng.normal(size=32 * 25)
    _, err = est.jackknife(x, np.mean, 32)
    means = x.reshape(32, 25).mean(axis=1)
    se = means.std(ddof=1) / math.sqrt(32)
    assert err == pytest.approx(se, rel=1e-12)


def test_c_function_reproduces_cylinder_cft():
    L = 2000
    for l in (100, 500, 1000, 1500):
        ds = est.cft_delta_s2(L, l)
        x = (l + 0.5) / L
        assert est.c_function(ds, 2, L, l) == pytest.approx(math.cos(math.pi * x) / 16,
                                                            abs=1e-6)


def test_c_function_normalisation_3d():
    # |dA| = 2L in 3D and the arc-length enters squared
    L, l, ds = 16, 3, 0.7
    x = (l + 0.5) / L
    assert est.c_function(ds, 3, L, l) == pytest.approx(
        (L / math.pi * math.sin(math.pi * x)) ** 2 * ds / (2 * L), rel=1e-15)


def test_increment_trick_is_running_sum():
    np.testing.assert_allclose(est.entropy_increments([0.5, 0.25, -0.1]),
                               [0.0, 0.5, 0.75, 0.65], atol=1e-15)
