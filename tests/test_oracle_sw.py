"""Pins of the oracle's Swendsen-Wang trajectories (the C program, update 1).

The paper's GPU code updates the replica lattice with Swendsen-Wang cluster
moves (section 3): every link of coupling K between equal spins becomes a bond
with probability 1 - e^{-2K}, and each cluster of bonded sites flips with
probability 1/2.  Along a transformation the switched column's self and glued
links carry the couplings beta (1 - lambda) and beta lambda.

* The exact Swendsen-Wang transition matrix (enumeration of all bond sets) is
  a stochastic matrix in detailed balance with the Boltzmann weight of every
  lambda, and its exact path measure satisfies Jarzynski's equality (eq. 2.9)
  to rounding.
* The joint law of (W_int, final energy) over many oracle trajectories matches
  that exact path measure, forward and reverse; each planted mistake (oracle
  built with ORACLE_MUTANT = 8..12) fails it.
* After thermalisation at a fixed geometry the oracle's (energy,
  magnetisation) law on 16-site lattices (2D and 3D) matches exact Boltzmann
  enumeration.
* Delta S_2 from Swendsen-Wang trajectories agrees with the exact
  transfer-matrix value; direct and reverse agree (Appendix A).
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
BETA_3D = 0.22165455
SW = 1

# (d, L, L_t, l, N, n_sweep, n_therm, direction); the exact kernel enumerates
# 2^18 bond sets of the 8-site replica lattice 2D L = L_t = 2
CASES = [(2, 2, 2, 1, 3, 1, 2, 1), (2, 2, 2, 0, 2, 2, 1, -1), (2, 2, 2, 1, 2, 1, 1, -1)]


def test_bond_threshold_special_values():
    assert oracle.bond_threshold(0.0) == 0                    # K = 0: never a bond
    assert oracle.bond_threshold(60.0) == 2 ** 32 - 1         # saturated
    for x in (1e-6, 0.3, 2 * BETA_2D, 5.0):
        T = oracle.bond_threshold(x)
        assert abs(T / 2.0 ** 32 - (1.0 - math.exp(-x))) <= 2.0 ** -32
    xs = np.linspace(0.0, 4.0, 41)
    assert all(np.diff([oracle.bond_threshold(float(x)) for x in xs]) > 0)


@functools.lru_cache(maxsize=None)
def _exact_joint(case):
    d, L, L_t, l, N, ns, nth, dirn = case
    wv, F = ex.exact_path_measure_sw(d, L, L_t, l, BETA_2D, N, ns, nth, direction=dirn)
    dyn = ex._SWDynamics(d, L, L_t, l, BETA_2D, N, dirn, True)
    e_final = dyn.energy(1.0).astype(np.int64)
    e_vals, e_idx = np.unique(e_final, return_inverse=True)
    P = np.zeros((len(wv), len(e_vals)))
    for j in range(len(e_vals)):
        P[:, j] = F[:, e_idx == j].sum(axis=1)
    return wv, P, e_idx


def joint_law_pvalue(case, n_traj, lib=None, seed=5):
    d, L, L_t, l, N, ns, nth, dirn = case
    wv, P, e_idx = _exact_joint(case)
    W, S = oracle.run(d, L, L_t, BETA_2D, l, N, ns, n_traj, seed, n_therm=nth, direction=dirn,
                      want_spins=True, lib=lib, update=SW)
    flat = S.reshape(n_traj, -1)
    state = ((flat < 0).astype(np.int64) << np.arange(flat.shape[1])).sum(axis=1)
    O = np.zeros_like(P)
    inside = np.abs(W) <= len(wv) // 2
    np.add.at(O, (W[inside] + len(wv) // 2, e_idx[state[inside]]), 1)
    expect = P * n_traj
    keep = expect > 5
    chi2 = float(((O[keep] - expect[keep]) ** 2 / expect[keep]).sum())
    stray = float(O[~keep].sum()) + float((~inside).sum())
    dof = int(keep.sum()) - 1
    return 1 - stats.chi2.cdf(chi2, dof), stray, float(expect[~keep].sum())


def test_exact_kernel_is_stochastic_and_in_detailed_balance():
    N = 3
    dyn = ex._SWDynamics(2, 2, 2, 1, BETA_2D, N, 1, False)
    for k, lam in [(None, 0.0), (0, 1.0 / 3.0), (2, 1.0)]:
        T = dyn.kernel(k)
        assert np.all(T >= 0)
        np.testing.assert_allclose(T.sum(axis=1), 1.0, atol=1e-12)
        e = -BETA_2D * dyn.energy(lam)
        pi = np.exp(e - e.max())
        pi /= pi.sum()
        D = pi[:, None] * T
        np.testing.assert_allclose(D, D.T, atol=1e-15)
    # flipping every spin is a symmetry of the update
    T = dyn.kernel(0)
    flip = (1 << dyn.V) - 1
    idx = np.arange(1 << dyn.V)
    np.testing.assert_allclose(T, T[np.ix_(idx ^ flip, idx ^ flip)], atol=1e-15)


@pytest.mark.parametrize("direction", [1, -1])
def test_exact_path_measure_satisfies_jarzynski(direction):
    d, L, L_t, l, N = 2, 2, 2, 1, 3
    w, F = ex.exact_path_measure_sw(d, L, L_t, l, BETA_2D, N, 1, 0, direction=direction,
                                    quantised=False, start="equilibrium")
    lhs = float(np.sum(F.sum(axis=1) * np.exp(-BETA_2D * w / N)))
    dlz = ex.log_z_enumerate(d, L, L_t, l, BETA_2D, lam=1.0) - \
        ex.log_z_enumerate(d, L, L_t, l, BETA_2D, lam=0.0)
    assert lhs == pytest.approx(math.exp(direction * dlz), rel=1e-12)


@pytest.mark.parametrize("case", CASES)
def test_work_and_energy_law_matches_exact_path_measure(case):
    p, stray, stray_expected = joint_law_pvalue(case, 100_000)
    assert p > 1e-4
    assert stray <= stray_expected + 6 * math.sqrt(stray_expected + 1)


@pytest.mark.parametrize("mutant", range(8, 13))
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


def _boltzmann_e_m(d, L, L_t, l, beta, lam):
    lk = ex.replica_links(d, L, L_t, l)
    sig = ex._spins_of_states(lk.n_sites).astype(np.int64)
    e = -(ex._bond_sums(sig, lk.full) + (1 - lam) * ex._bond_sums(sig, lk.self_)
          + lam * ex._bond_sums(sig, lk.glue))
    m = sig.sum(axis=1)
    w = np.exp(-beta * (e - e.min()))
    return np.rint(e).astype(np.int64), m, w / w.sum()


@pytest.mark.parametrize("d,L,L_t,l,beta,direction",
                         [(2, 4, 2, 1, BETA_2D, 1), (2, 2, 4, 0, BETA_2D, -1),
                          (3, 2, 2, 1, BETA_3D, 1)])
def test_thermalised_state_follows_boltzmann(d, L, L_t, l, beta, direction):
    # no protocol sweeps: the final state is the one after n_therm updates at
    # the start geometry (lambda = 0 forward, 1 reverse)
    lam = 0.0 if direction > 0 else 1.0
    e, m, pi = _boltzmann_e_m(d, L, L_t, l, beta, lam)
    n = 60_000
    _, S = oracle.run(d, L, L_t, beta, l, 1, 0, n, 17, n_therm=12, direction=direction,
                      want_spins=True, update=SW)
    flat = S.reshape(n, -1).astype(np.int64)
    state = ((flat < 0).astype(np.int64) << np.arange(flat.shape[1])).sum(axis=1)
    keys = e * 1000 + m
    uk, inv = np.unique(keys, return_inverse=True)
    P = np.bincount(inv, weights=pi, minlength=len(uk))
    O = np.bincount(inv[state], minlength=len(uk)).astype(float)
    expect = P * n
    keep = expect > 5
    chi2 = float(((O[keep] - expect[keep]) ** 2 / expect[keep]).sum())
    assert 1 - stats.chi2.cdf(chi2, int(keep.sum()) - 1) > 1e-4
    assert O[~keep].sum() <= expect[~keep].sum() + 6 * math.sqrt(expect[~keep].sum() + 1)


@pytest.mark.parametrize("d,L,L_t,l", [(2, 4, 8, 2), (3, 2, 4, 0)])
def test_delta_s2_agrees_with_transfer_matrix(d, L, L_t, l):
    beta = BETA_2D if d == 2 else BETA_3D
    exact = ex.delta_s2_transfer(d, L, L_t, beta)[l]
    W, _ = oracle.run(d, L, L_t, beta, l, 20, 1, 4000, 13, n_therm=20, update=SW)
    val, err = est.delta_s2_with_error(W, beta, 20)
    assert abs(val - exact) < 4 * err + 1e-3 * abs(exact)
    assert err < 0.05 * abs(exact) + 0.005


def test_direct_and_reverse_agree():
    d, L, L_t, l, N = 2, 6, 6, 2, 30
    Wf, _ = oracle.run(d, L, L_t, BETA_2D, l, N, 1, 3000, 6, n_therm=30, direction=1, update=SW)
    Wr, _ = oracle.run(d, L, L_t, BETA_2D, l, N, 1, 3000, 6, n_therm=30, direction=-1, update=SW)
    vf, ef = est.delta_s2_with_error(Wf, BETA_2D, N, 1)
    vr, er = est.delta_s2_with_error(Wr, BETA_2D, N, -1)
    assert abs(vf - vr) < 4 * math.hypot(ef, er)


def test_thread_count_and_range_split_do_not_matter():
    args = (3, 4, 4, BETA_3D, 1, 5, 2, 20, 7)
    W1, S1 = oracle.run(*args, n_therm=4, n_threads=1, want_spins=True, update=SW)
    W4, S4 = oracle.run(*args, n_therm=4, n_threads=4, want_spins=True, update=SW)
    np.testing.assert_array_equal(W1, W4)
    np.testing.assert_array_equal(S1, S4)
    d, L, L_t, beta, l, N, ns, n, seed = args
    Wa, Sa = oracle.run(d, L, L_t, beta, l, N, ns, 8, seed, n_therm=4, traj0=12,
                        want_spins=True, update=SW)
    np.testing.assert_array_equal(Wa, W1[12:20])
    np.testing.assert_array_equal(Sa, S1[12:20])


def test_update_selects_a_different_chain():
    args = (2, 8, 8, BETA_2D, 3, 6, 1, 16, 1)
    Wm, Sm = oracle.run(*args, n_therm=5, want_spins=True, update=0)
    Ws, Ss = oracle.run(*args, n_therm=5, want_spins=True, update=SW)
    assert not np.array_equal(Sm, Ss)
    with pytest.raises(ValueError):
        oracle.run(*args, n_therm=5, update=2)
