"""Pins of the oracle's Monte Carlo trajectories (the C program).

* The joint law of (W_int, final energy) over many trajectories matches the
  exact path measure of the same dynamics (hot start, n_therm sweeps at the start
  geometry, work before each update, update at lambda_{k+1}: Appendix A),
  forward and reverse, 2D and 3D.
* Each planted mistake (oracle built with ORACLE_MUTANT = 1..7) fails that test.
* The Jarzynski estimate of Delta S_2 agrees with the exact transfer-matrix
  value within its jackknife error; direct and reverse agree (Appendix A, eq.
  equality_of_direct_reverse_protocols); beta = 0 gives Delta S_2 = 0 exactly.
* Trajectories are independent: results do not depend on the thread count or on
  how the trajectory range is split.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle
import oracle.estimator as est
import oracle.exact as ex

BETA_2D = 0.5 * math.log(1 + math.sqrt(2))

# (d, L, L_t, l, N, n_sweep, n_therm, direction)
CASES = [(2, 2, 4, 1, 3, 1, 5, 1), (2, 4, 2, 1, 2, 2, 3, 1), (2, 4, 2, 2, 2, 1, 3, -1),
         (3, 2, 2, 1, 3, 1, 4, 1)]


def joint_law_pvalue(case, n_traj, lib=None, seed=3):
    d, L, L_t, l, N, ns, nth, dirn = case
    wv, F = ex.exact_path_measure(d, L, L_t, l, BETA_2D, N, ns, nth, direction=dirn)
    dyn = ex._Dynamics(d, L, L_t, l, BETA_2D, N, dirn, True)
    e_final = dyn.energy(1.0).astype(np.int64)
    e_vals, e_idx = np.unique(e_final, return_inverse=True)
    P = np.zeros((len(wv), len(e_vals)))
    for j in range(len(e_vals)):
        P[:, j] = F[:, e_idx == j].sum(axis=1)
    W, S = oracle.run(d, L, L_t, BETA_2D, l, N, ns, n_traj, seed, n_therm=nth, direction=dirn,
                      want_spins=True, lib=lib)
    flat = S.reshape(n_traj, -1)
    state = ((flat < 0).astype(np.int64) << np.arange(flat.shape[1])).sum(axis=1)
    O = np.zeros_like(P)
    np.add.at(O, (W + len(wv) // 2, e_idx[state]), 1)
    expect = P * n_traj
    keep = expect > 5
    chi2 = float(((O[keep] - expect[keep]) ** 2 / expect[keep]).sum())
    # mass where the exact law has (almost) none also counts against the oracle
    stray = float(O[~keep].sum())
    dof = int(keep.sum()) - 1
    return 1 - stats.chi2.cdf(chi2, dof), stray, float(expect[~keep].sum())


@pytest.mark.parametrize("case", CASES)
def test_work_and_energy_law_matches_exact_path_measure(case):
    p, stray, stray_expected = joint_law_pvalue(case, 100_000)
    assert p > 1e-4
    assert stray <= stray_expected + 6 * math.sqrt(stray_expected + 1)


@pytest.mark.parametrize("mutant", range(1, 8))
def test_planted_mistakes_are_caught(mutant, tmp_path):
    path = oracle.build(out=str(tmp_path / f"liboracle_m{mutant}.so"), mutant=mutant)
    lib = oracle.load_library(path)
    worst = 1.0
    for case in CASES:
        p, stray, stray_expected = joint_law_pvalue(case, 100_000, lib=lib)
        if stray > stray_expected + 6 * math.sqrt(stray_expected + 1):
            p = 0.0
        worst = min(worst, p)
    assert worst < 1e-8


@pytest.mark.parametrize("d,L,L_t,l", [(2, 4, 4, 1), (2, 4, 8, 2), (3, 2, 4, 0)])
def test_delta_s2_agrees_with_transfer_matrix(d, L, L_t, l):
    beta = BETA_2D if d == 2 else 0.22165455
    exact = ex.delta_s2_transfer(d, L, L_t, beta)[l]
    W, _ = oracle.run(d, L, L_t, beta, l, 20, 1, 4000, 11, n_therm=200)
    val, err = est.delta_s2_with_error(W, beta, 20)
    assert abs(val - exact) < 4 * err + 1e-3 * abs(exact)
    assert err < 0.05 * abs(exact) + 0.005


def test_direct_and_reverse_agree():
    d, L, L_t, l, N = 2, 6, 6, 2, 30
    Wf, _ = oracle.run(d, L, L_t, BETA_2D, l, N, 1, 3000, 5, n_therm=300, direction=1)
    Wr, _ = oracle.run(d, L, L_t, BETA_2D, l, N, 1, 3000, 5, n_therm=300, direction=-1)
    vf, ef = est.delta_s2_with_error(Wf, BETA_2D, N, 1)
    vr, er = est.delta_s2_with_error(Wr, BETA_2D, N, -1)
    assert abs(vf - vr) < 4 * math.hypot(ef, er)
    # the two directions really are different runs
    assert not np.array_equal(Wf, -Wr)


def test_beta_zero_gives_zero_entropy_change():
    W, _ = oracle.run(2, 8, 8, 0.0, 3, 10, 1, 64, 2, n_therm=5)
    assert est.delta_s2(W, 0.0, 10) == 0.0
    assert np.any(W != 0)          # the integer work itself still fluctuates


def test_thread_count_and_range_split_do_not_matter():
    args = (2, 8, 8, BETA_2D, 3, 7, 2, 24, 99)
    W1, S1 = oracle.run(*args, n_therm=9, n_threads=1, want_spins=True)
    W4, S4 = oracle.run(*args, n_therm=9, n_threads=4, want_spins=True)
    np.testing.assert_array_equal(W1, W4)
    np.testing.assert_array_equal(S1, S4)
    d, L, L_t, beta, l, N, ns, n, seed = args
    Wa, Sa = oracle.run(d, L, L_t, beta, l, N, ns, 10, seed, n_therm=9, traj0=14,
                        want_spins=True)
    np.testing.assert_array_equal(Wa, W1[14:24])
    np.testing.assert_array_equal(Sa, S1[14:24])


def test_seed_and_l_select_distinct_streams():
    W0, S0 = oracle.run(2, 8, 8, BETA_2D, 3, 5, 1, 8, 1, n_therm=3, want_spins=True)
    W1, S1 = oracle.run(2, 8, 8, BETA_2D, 3, 5, 1, 8, 2, n_therm=3, want_spins=True)
    W2, S2 = oracle.run(2, 8, 8, BETA_2D, 4, 5, 1, 8, 1, n_therm=3, want_spins=True)
    assert not np.array_equal(S0, S1)
    assert not np.array_equal(S0, S2)


def test_spins_are_plus_minus_one_and_work_bounded():
    N = 6
    W, S = oracle.run(3, 4, 4, 0.22165455, 1, N, 1, 16, 4, n_therm=4, want_spins=True)
    assert set(np.unique(S)) <= {-1, 1}
    # |dE_k| <= 2 n L^(d-2) and dE_k is even
    assert np.all(np.abs(W) <= 2 * 2 * 4 * N)
    assert np.all(W % 2 == 0)


@pytest.mark.parametrize("bad", [dict(d=4), dict(L=5), dict(L_t=3), dict(l=8), dict(l=-1),
                                 dict(n_step=0), dict(direction=0)])
def test_rejects_bad_arguments(bad):
    kw = dict(d=2, L=8, L_t=8, beta=0.4, l=2, n_step=4, n_sweep=1, n_traj=2, seed=0)
    direction = bad.pop("direction", 1)
    kw.update(bad)
    with pytest.raises(ValueError):
        oracle.run(kw["d"], kw["L"], kw["L_t"], kw["beta"], kw["l"], kw["n_step"],
                   kw["n_sweep"], kw["n_traj"], kw["seed"], n_therm=1, direction=direction)


def test_thresholds_match_boltzmann_factor():
    for beta in (0.1, BETA_2D, 1.0):
        for m in (2, 4, 6):
            T = oracle.threshold_bulk(beta, m)
            assert abs(T / 2.0 ** 32 - math.exp(-2 * beta * m)) <= 2.0 ** -32
        for N in (1, 7, 1000):
            for m in (1, 5, 3 * N + 1):
                T = oracle.threshold_cut(beta, m, N)
                assert abs(T / 2.0 ** 32 - math.exp(-2 * beta * m / N)) <= 2.0 ** -32
    # e^0 = 1 would give 2^32: the threshold saturates at 2^32 - 1
    assert oracle.threshold_bulk(0.0, 2) == 2 ** 32 - 1
    assert oracle.threshold_cut(0.0, 5, 3) == 2 ** 32 - 1
    # far past the range of exp, the threshold is 0 (never flips for m > 0)
    assert oracle.threshold_bulk(40.0, 6) == 0
