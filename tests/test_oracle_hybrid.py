"""Pins of the oracle's thermalisation option: Swendsen-Wang sweeps for the
start, Metropolis sweeps for the protocol (therm_update = 1).

Appendix A's identity <e^-W> = Z(lambda_N)/Z(lambda_0) needs an equilibrium
start and protocol sweeps that keep each step's Boltzmann weight; section 4
thermalises with cluster steps.  The oracle composes its two pinned updates:

* Joint law of (W_int, final energy) over many oracle trajectories against the
  exact path measure of a hot start, n_therm exact Swendsen-Wang steps and the
  exact Metropolis protocol (2D L = L_t = 2, enumeration of all 256 states),
  forward and reverse, for a moving end of region A and a whole cut.  The
  same trajectories with Metropolis thermalisation
  fail it: from a hot start one or two steps of the two updates leave
  different laws.
* With no thermalisation sweeps the option changes nothing (bit for bit).
* With no protocol sweeps the final state is the Swendsen-Wang run's final
  state (bit for bit): the thermalisation sweeps take the Swendsen-Wang random
  stream of sweep indices 0 .. n_therm-1.
* Delta S_2 agrees with the exact transfer-matrix value.
"""
import functools
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import oracle.estimator as est
import oracle.exact as ex

BETA_2D = 0.5 * math.log(1 + math.sqrt(2))
SW = 1

# (d, L, L_t, l, N, n_sweep, n_therm, direction)
CASES = [(2, 2, 2, 1, 3, 1, 1, 1), (2, 2, 2, 0, 2, 2, 2, -1)]


@functools.lru_cache(maxsize=None)
def _exact_joint(case, therm, whole=False):
    d, L, L_t, l, N, ns, nth, dirn = case
    wv, F = ex.exact_path_measure(d, L, L_t, l, BETA_2D, N, ns, nth, direction=dirn,
                                  therm=therm, whole=whole)
    dyn = ex._Dynamics(d, L, L_t, l, BETA_2D, N, dirn, True, 1, 2, whole)
    e_vals, e_idx = np.unique(dyn.energy(1.0).astype(np.int64), return_inverse=True)
    P = np.zeros((len(wv), len(e_vals)))
    for j in range(len(e_vals)):
        P[:, j] = F[:, e_idx == j].sum(axis=1)
    return wv, P, e_idx


def _pvalue(case, therm_update, exact_therm, n_traj=100_000, seed=9, whole=False):
    d, L, L_t, l, N, ns, nth, dirn = case
    wv, P, e_idx = _exact_joint(case, exact_therm, whole)
    W, S = oracle.run(d, L, L_t, BETA_2D, l, N, ns, n_traj, seed, n_therm=nth, direction=dirn,
                      want_spins=True, therm_update=therm_update, whole=whole)
    flat = S.reshape(n_traj, -1)
    state = ((flat < 0).astype(np.int64) << np.arange(flat.shape[1])).sum(axis=1)
    O = np.zeros_like(P)
    inside = np.abs(W) <= len(wv) // 2
    np.add.at(O, (W[inside] + len(wv) // 2, e_idx[state[inside]]), 1)
    expect = P * n_traj
    keep = expect > 5
    chi2 = float(((O[keep] - expect[keep]) ** 2 / expect[keep]).sum())
    stray = float(O[~keep].sum()) + float((~inside).sum())
    return 1 - stats.chi2.cdf(chi2, int(keep.sum()) - 1), stray, float(expect[~keep].sum())


def test_exact_laws_of_the_two_thermalisations_differ():
    for case in CASES:
        _, Pm, _ = _exact_joint(case, "metropolis")
        _, Ps, _ = _exact_joint(case, "sw")
        assert np.abs(Pm - Ps).sum() > 0.01


@pytest.mark.parametrize("case", CASES)
def test_joint_law_matches_exact_path_measure(case):
    p, stray, stray_expected = _pvalue(case, SW, "sw")
    assert p > 1e-4
    assert stray <= stray_expected + 6 * math.sqrt(stray_expected + 1)


@pytest.mark.parametrize("direction", [1, -1])
def test_whole_cut_joint_law_matches_exact_path_measure(direction):
    """The whole-cut transformation (both columns of 2D L = 2 switch from
    decoupled to glued replicas) from a Swendsen-Wang start."""
    case = (2, 2, 2, 2, 3, 1, 1, direction)
    p, stray, stray_expected = _pvalue(case, SW, "sw", whole=True)
    assert p > 1e-4
    assert stray <= stray_expected + 6 * math.sqrt(stray_expected + 1)


@pytest.mark.parametrize("case", CASES)
def test_metropolis_thermalisation_fails_the_same_law(case):
    p, _, _ = _pvalue(case, 0, "sw")
    assert p < 1e-6


def test_no_thermalisation_sweeps_change_nothing():
    for d, L, L_t, l in [(2, 6, 4, 2), (3, 4, 4, 1)]:
        a = oracle.run(d, L, L_t, 0.4, l, 5, 2, 7, 3, n_therm=0, want_spins=True,
                       therm_update=SW)
        b = oracle.run(d, L, L_t, 0.4, l, 5, 2, 7, 3, n_therm=0, want_spins=True)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


def test_thermalised_state_is_the_swendsen_wang_one():
    """n_sweep = 0: no protocol sweep, so the final state is the thermalised
    one, and W_int = N dE_0 on it."""
    for d, L, L_t, l, dirn in [(2, 6, 4, 2, 1), (3, 4, 4, 1, -1)]:
        hyb = oracle.run(d, L, L_t, 0.4, l, 3, 0, 9, 11, n_therm=5, direction=dirn,
                         want_spins=True, therm_update=SW)
        sw = oracle.run(d, L, L_t, 0.4, l, 3, 0, 9, 11, n_therm=5, direction=dirn,
                        want_spins=True, update=SW)
        met = oracle.run(d, L, L_t, 0.4, l, 3, 0, 9, 11, n_therm=5, direction=dirn,
                         want_spins=True)
        np.testing.assert_array_equal(hyb[1], sw[1])
        np.testing.assert_array_equal(hyb[0], sw[0])
        assert not np.array_equal(hyb[1], met[1])


def test_delta_s2_agrees_with_transfer_matrix():
    d, L, L_t, l = 2, 4, 4, 1
    exact = ex.delta_s2_transfer(d, L, L_t, BETA_2D)[l]
    W, _ = oracle.run(d, L, L_t, BETA_2D, l, 40, 1, 20000, 21, n_therm=20, therm_update=SW)
    ds, err = est.delta_s2_with_error(W, BETA_2D, 40, 1, 32)
    assert abs(ds - exact) <= 4.5 * err + 1e-3
