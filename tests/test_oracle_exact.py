"""Pins of the oracle's exact solvers against closed forms and each other.

* Kaufman's finite-torus Z (closed form) == brute-force enumeration.
* Replica transfer matrix == brute-force enumeration of the replica lattice.
* Fully glued replicas form one torus of doubled time: Z_2(l = L) = Z(L, 2 L_t);
  Z_2(0) = Z(L, L_t)^2 (section 2: Tr rho^n = Z_n / Z^n).
* Geometry l at lambda = 1 is geometry l+1 at lambda = 0 (section 3 protocol).
* The cylinder CFT form of section 2 and the 2D fit of section 4
  (C_2 = cos(pi x)/16 + k cot(pi x)/(2L)) at L_t = 8L, and the zero-temperature
  symmetry C(x) = -C(1-x) improving with L_t (section 4).
* The exact Jarzynski identity <e^-W> = Z_f/Z_i of Appendix A for any N, and its
  failure when the update uses lambda_k instead of lambda_{k+1}.
"""
import math

import numpy as np
import pytest

import oracle.estimator as est
import oracle.exact as ex

BETA_2D = 0.5 * math.log(1 + math.sqrt(2))


@pytest.mark.parametrize("m,n", [(2, 2), (2, 4), (4, 4), (4, 2), (2, 6), (4, 3), (3, 4)])
@pytest.mark.parametrize("beta", [0.1, BETA_2D, 0.8])
def test_kaufman_equals_enumeration(m, n, beta):
    assert ex.log_z_kaufman(m, n, beta) == pytest.approx(
        ex.log_z_single_enumerate(2, n, m, beta), abs=1e-11)


@pytest.mark.parametrize("d,L,L_t", [(2, 2, 4), (2, 4, 2), (3, 2, 2)])
@pytest.mark.parametrize("beta", [0.2, BETA_2D])
def test_transfer_matrix_equals_enumeration(d, L, L_t, beta):
    ls = list(range(L + 1))
    lz_t = ex.log_z2_transfer(d, L, L_t, ls, beta)
    lz_e = np.array([ex.log_z_enumerate(d, L, L_t, l, beta) if l < L else
                     ex.log_z_enumerate(d, L, L_t, L - 1, beta, lam=1.0) for l in ls])
    np.testing.assert_allclose(np.diff(lz_t), np.diff(lz_e), atol=1e-11)


@pytest.mark.parametrize("d,L,L_t", [(2, 2, 4), (2, 4, 2), (3, 2, 2)])
def test_lambda_one_is_next_geometry(d, L, L_t):
    for l in range(L - 1):
        assert ex.log_z_enumerate(d, L, L_t, l, 0.37, lam=1.0) == pytest.approx(
            ex.log_z_enumerate(d, L, L_t, l + 1, 0.37, lam=0.0), abs=1e-12)


@pytest.mark.parametrize("d,L,L_t", [(2, 2, 4), (2, 4, 2), (3, 2, 2)])
def test_replica_limits_by_enumeration(d, L, L_t):
    beta = 0.3
    z1 = ex.log_z_single_enumerate(d, L, L_t, beta)
    assert ex.log_z_enumerate(d, L, L_t, 0, beta) == pytest.approx(2 * z1, abs=1e-11)
    if 2 * L_t * L ** (d - 1) <= 16:
        z_double = ex.log_z_single_enumerate(d, L, 2 * L_t, beta)
        glued = ex.log_z_enumerate(d, L, L_t, L - 1, beta, lam=1.0)
        assert glued == pytest.approx(z_double, abs=1e-11)


@pytest.mark.parametrize("L,L_t", [(6, 8), (8, 16)])
def test_sum_of_increments_is_kaufman(L, L_t):
    """sum_l Delta S_2(l) = -ln[Z(L, 2 L_t) / Z(L, L_t)^2], exact in 2D."""
    ds = ex.delta_s2_transfer(2, L, L_t, BETA_2D)
    rhs = -(ex.log_z_kaufman(2 * L_t, L, BETA_2D) - 2 * ex.log_z_kaufman(L_t, L, BETA_2D))
    assert ds.sum() == pytest.approx(rhs, abs=1e-10)


def test_cft_and_first_correction_at_zero_temperature():
    """At L_t = 8L the exact C_2 follows cos(pi x)/16 + k cot(pi x)/(2L) on the
    interior points with k in the range the paper fits (section 4, table 1)."""
    L = 10
    ds = ex.delta_s2_transfer(2, L, 8 * L, BETA_2D)
    ls = np.arange(1, L - 1)
    x = (ls + 0.5) / L
    C = np.array([est.c_function(ds[l], 2, L, l) for l in ls])
    scaling = np.cos(np.pi * x) / 16
    corr = 1 / np.tan(np.pi * x) / (2 * L)
    k = float(np.sum((C - scaling) * corr) / np.sum(corr * corr))
    assert 0.12 < k < 0.22
    assert np.max(np.abs(C - scaling - k * corr)) < 3e-3
    # without the correction the data miss the scaling function badly
    assert np.max(np.abs(C - scaling)) > 5e-3


def test_zero_temperature_symmetry_improves_with_time_extent():
    """C(x) = -C(1-x) needs L_t >> L (section 4); Delta S_2(l) + Delta S_2(L-1-l)
    shrinks as L_t / L grows."""
    L = 8
    asym = []
    for ratio in (1, 2, 4, 8):
        ds = ex.delta_s2_transfer(2, L, ratio * L, BETA_2D)
        asym.append(max(abs(ds[l] + ds[L - 1 - l]) for l in range(L // 2)))
    assert all(a > b for a, b in zip(asym, asym[1:]))
    assert asym[-1] < 2e-3


@pytest.mark.parametrize("n_step", [1, 2, 3])
@pytest.mark.parametrize("direction", [1, -1])
def test_exact_jarzynski_identity(n_step, direction):
    """Sum over the exact path measure of e^{-W} equals Z_f / Z_i (Appendix A)."""
    d, L, L_t, l, beta = 2, 2, 4, 1, BETA_2D
    w, F = ex.exact_path_measure(d, L, L_t, l, beta, n_step, 1, 0, direction=direction,
                                 quantised=False, start="equilibrium")
    lhs = float(np.sum(F.sum(axis=1) * np.exp(-beta * w / n_step)))
    z0 = ex.log_z_enumerate(d, L, L_t, l, beta, lam=0.0)
    z1 = ex.log_z_enumerate(d, L, L_t, l, beta, lam=1.0)
    ratio = math.exp(z1 - z0) if direction > 0 else math.exp(z0 - z1)
    assert lhs == pytest.approx(ratio, rel=1e-12)
    # the 32-bit thresholds perturb the identity by no more than ~2^-32 per step
    w, F = ex.exact_path_measure(d, L, L_t, l, beta, n_step, 1, 0, direction=direction,
                                 quantised=True, start="equilibrium")
    lhs_q = float(np.sum(F.sum(axis=1) * np.exp(-beta * w / n_step)))
    assert lhs_q == pytest.approx(ratio, rel=1e-7)


def test_jarzynski_identity_needs_update_at_next_lambda(monkeypatch):
    """Updating step k with lambda_k (not lambda_{k+1}) breaks the identity:
    this pins the ordering remark after the discretised average in Appendix A."""
    d, L, L_t, l, beta, n_step = 2, 2, 4, 1, BETA_2D, 3
    orig = ex._Dynamics._flip_prob

    def lagged(self, i, k):
        return orig(self, i, None if k == 0 else (k - 1 if k is not None else None))
    monkeypatch.setattr(ex._Dynamics, "_flip_prob", lagged)
    w, F = ex.exact_path_measure(d, L, L_t, l, beta, n_step, 1, 0, quantised=False,
                                 start="equilibrium")
    lhs = float(np.sum(F.sum(axis=1) * np.exp(-beta * w / n_step)))
    ratio = math.exp(ex.log_z_enumerate(d, L, L_t, l, beta, lam=1.0)
                     - ex.log_z_enumerate(d, L, L_t, l, beta, lam=0.0))
    assert abs(lhs / ratio - 1) > 1e-4


def test_beta_zero_has_no_entropy_change():
    ds = ex.delta_s2_transfer(2, 4, 4, 0.0)
    np.testing.assert_allclose(ds, 0.0, atol=1e-13)
