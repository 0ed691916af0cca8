"""Pins of protocol 2 (Appendix B): the L_y switched columns of a 3D cut are
switched one after another, m = N/L_y steps each.

* The exact path measure of protocol 2 (every state of the 16-site 3D lattice
  L = L_t = 2) satisfies Jarzynski's equality to rounding, both directions, and
  its work law differs from protocol 1's (so the schedule really changes the
  dynamics while keeping the free-energy difference).
* The oracle's joint law of (W_int, final energy) with protocol 2 matches that
  exact path measure; the planted mistake 13 (work of the active column not
  scaled by L_y) fails it.
* In 2D (L_y = 1) protocol 2 is protocol 1: identical W and spins, both updates.
* Delta S_2 from protocol-2 trajectories agrees with the transfer matrix, for
  both updates; n_step not a multiple of L_y is rejected.
"""
import functools
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import oracle.estimator as est
import oracle.exact as ex

BETA_3D = 0.22165455

# (d, L, L_t, l, N, n_sweep, n_therm, direction)
CASES = [(3, 2, 2, 1, 4, 1, 3, 1), (3, 2, 2, 0, 2, 2, 2, -1)]


@pytest.mark.parametrize("direction", [1, -1])
def test_exact_protocol2_satisfies_jarzynski(direction):
    d, L, L_t, l, N = 3, 2, 2, 1, 4
    w, F = ex.exact_path_measure(d, L, L_t, l, BETA_3D, N, 1, 0, direction=direction,
                                 quantised=False, start="equilibrium", protocol=2)
    lhs = float(np.sum(F.sum(axis=1) * np.exp(-BETA_3D * w / N)))
    dlz = ex.log_z_enumerate(d, L, L_t, l, BETA_3D, lam=1.0) - \
        ex.log_z_enumerate(d, L, L_t, l, BETA_3D, lam=0.0)
    assert lhs == pytest.approx(math.exp(direction * dlz), rel=1e-12)


def test_protocols_have_different_work_laws():
    args = (3, 2, 2, 1, BETA_3D, 4, 1, 2)
    w1, F1 = ex.exact_path_measure(*args, protocol=1)
    w2, F2 = ex.exact_path_measure(*args, protocol=2)
    assert np.array_equal(w1, w2)
    p1, p2 = F1.sum(axis=1), F2.sum(axis=1)
    assert np.abs(p1 - p2).sum() > 0.1
    # protocol 2's work comes in multiples of L_y = 2 times the pair sums
    assert np.all(p2[(w2 % 4) != 0] < 1e-15)


@functools.lru_cache(maxsize=None)
def _exact_joint(case):
    d, L, L_t, l, N, ns, nth, dirn = case
    wv, F = ex.exact_path_measure(d, L, L_t, l, BETA_3D, N, ns, nth, direction=dirn,
                                  protocol=2)
    dyn = ex._Dynamics(d, L, L_t, l, BETA_3D, N, dirn, True, 2)
    e_vals, e_idx = np.unique(dyn.energy(1.0).astype(np.int64), return_inverse=True)
    P = np.zeros((len(wv), len(e_vals)))
    for j in range(len(e_vals)):
        P[:, j] = F[:, e_idx == j].sum(axis=1)
    return wv, P, e_idx


def joint_law_pvalue(case, n_traj, lib=None, seed=9):
    d, L, L_t, l, N, ns, nth, dirn = case
    wv, P, e_idx = _exact_joint(case)
    W, S = oracle.run(d, L, L_t, BETA_3D, l, N, ns, n_traj, seed, n_therm=nth, direction=dirn,
                      want_spins=True, lib=lib, protocol=2)
    flat = S.reshape(n_traj, -1)
    state = ((flat < 0).astype(np.int64) << np.arange(flat.shape[1])).sum(axis=1)
    O = np.zeros_like(P)
    inside = np.abs(W) <= len(wv) // 2
    np.add.at(O, (W[inside] + len(wv) // 2, e_idx[state[inside]]), 1)
    expect = P * n_traj
    keep = expect > 5
    chi2 = float(((O[keep] - expect[keep]) ** 2 / expect[keep]).sum())
    stray = float(O[~keep].sum()) + float((~inside).sum())
    return (1 - stats.chi2.cdf(chi2, int(keep.sum()) - 1), stray,
            float(expect[~keep].sum()))


@pytest.mark.parametrize("case", CASES)
def test_protocol2_law_matches_exact_path_measure(case):
    p, stray, stray_expected = joint_law_pvalue(case, 100_000)
    assert p > 1e-4
    assert stray <= stray_expected + 6 * math.sqrt(stray_expected + 1)


def test_unscaled_work_is_caught(tmp_path):
    lib = oracle.load_library(oracle.build(out=str(tmp_path / "liboracle_m13.so"), mutant=13))
    p, stray, stray_expected = joint_law_pvalue(CASES[0], 100_000, lib=lib)
    assert p < 1e-8 or stray > stray_expected + 6 * math.sqrt(stray_expected + 1)


@pytest.mark.parametrize("update", [0, 1])
def test_protocol2_is_protocol1_in_2d(update):
    args = (2, 8, 8, 0.44, 3, 12, 2, 16, 5)
    W1, S1 = oracle.run(*args, n_therm=4, want_spins=True, update=update, protocol=1)
    W2, S2 = oracle.run(*args, n_therm=4, want_spins=True, update=update, protocol=2)
    np.testing.assert_array_equal(W1, W2)
    np.testing.assert_array_equal(S1, S2)


@pytest.mark.parametrize("update", [0, 1])
def test_protocol2_delta_s2_agrees_with_transfer_matrix(update):
    d, L, L_t, l, N = 3, 2, 4, 0, 20
    exact = ex.delta_s2_transfer(d, L, L_t, BETA_3D)[l]
    W, _ = oracle.run(d, L, L_t, BETA_3D, l, N, 1, 4000, 21, n_therm=40, update=update,
                      protocol=2)
    assert np.all(W % 2 == 0)
    val, err = est.delta_s2_with_error(W, BETA_3D, N)
    assert abs(val - exact) < 4 * err + 1e-3 * abs(exact)


def test_protocol2_needs_whole_runs_per_column():
    with pytest.raises(ValueError):
        oracle.run(3, 4, 4, BETA_3D, 1, 6, 1, 2, 0, n_therm=1, protocol=2)
    with pytest.raises(ValueError):
        oracle.run(3, 4, 4, BETA_3D, 1, 8, 1, 2, 0, n_therm=1, protocol=3)
