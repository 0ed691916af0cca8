"""Pins of the n-replica geometry (section 2, S_n = ln(Z_n/Z^n)/(1-n)) and of
Alba et al.'s whole-cut transformation (section 3: every coupling across a cut
of length l switches together, from n decoupled replicas to glued ones).

* The n-replica transfer matrix Z_n(l) = Tr M_l^n equals enumeration (n = 3, 4);
  fully glued replicas are one lattice of extent n L_t (Kaufman), so
  ln Z_n(L) - n ln Z = ln Z(L, n L_t) - n ln Z(L, L_t); S_n(0) = 0.
* The exact path measures of the n = 3 transformation and of the whole-cut
  transformation satisfy Jarzynski's equality to rounding, both directions.
* The oracle's joint law of (W_int, final energy) matches those exact path
  measures; planted mistakes (no glue, sign of the work) fail it.
* Delta S_3 and the whole-cut S_2(l), S_3(l) from Monte Carlo agree with the
  transfer matrix, for both updates.
"""
import functools
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import oracle.estimator as est
import oracle.exact as ex

BETA = 0.5 * math.log(1 + math.sqrt(2))


@pytest.mark.parametrize("n", [3, 4])
def test_n_replica_transfer_matrix_equals_enumeration(n):
    d, L, L_t = 2, 2, 2
    lz = ex.log_zn_transfer(d, L, L_t, range(L + 1), BETA, n)
    en = [ex.log_z_enumerate(d, L, L_t, l, BETA, lam=0.0, n=n) for l in range(L)]
    en.append(ex.log_z_enumerate(d, L, L_t, L - 1, BETA, lam=1.0, n=n))
    np.testing.assert_allclose(lz - lz[0], np.array(en) - en[0], atol=1e-12)
    # the whole-cut geometry at lambda = 0 is n decoupled lattices
    z1 = ex.log_z_single_enumerate(d, L, L_t, BETA)
    assert ex.log_z_enumerate(d, L, L_t, L, BETA, lam=0.0, n=n, whole=True) == \
        pytest.approx(n * z1, abs=1e-12)


@pytest.mark.parametrize("n", [2, 3, 5])
@pytest.mark.parametrize("L,L_t", [(4, 4), (6, 2)])
def test_fully_glued_replicas_form_one_long_lattice(n, L, L_t):
    s = ex.renyi_sn_transfer(2, L, L_t, BETA, n)
    assert s[0] == 0.0
    want = (ex.log_z_kaufman(L, n * L_t, BETA) - n * ex.log_z_kaufman(L, L_t, BETA)) / (1 - n)
    assert s[-1] == pytest.approx(want, rel=1e-10)
    # the increments telescope to the whole-cut entropy
    ds = ex.delta_sn_transfer(2, L, L_t, BETA, n)
    np.testing.assert_allclose(np.cumsum(ds), s[1:], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("whole,l", [(False, 1), (True, 2), (True, 1)])
@pytest.mark.parametrize("direction", [1, -1])
def test_exact_n3_and_whole_cut_satisfy_jarzynski(whole, l, direction):
    d, L, L_t, n, N = 2, 2, 2, 3, 3
    w, F = ex.exact_path_measure(d, L, L_t, l, BETA, N, 1, 0, direction=direction,
                                 quantised=False, start="equilibrium", n=n, whole=whole)
    lhs = float(np.sum(F.sum(axis=1) * np.exp(-BETA * w / N)))
    dlz = ex.log_z_enumerate(d, L, L_t, l, BETA, lam=1.0, n=n, whole=whole) - \
        ex.log_z_enumerate(d, L, L_t, l, BETA, lam=0.0, n=n, whole=whole)
    assert lhs == pytest.approx(math.exp(direction * dlz), rel=1e-12)


# (d, L, L_t, l, N, n_sweep, n_therm, direction, n, whole)
CASES = [(2, 2, 2, 1, 3, 1, 3, 1, 3, False), (2, 2, 2, 0, 2, 2, 2, -1, 3, False),
         (2, 2, 2, 2, 3, 1, 3, 1, 3, True), (2, 2, 2, 1, 2, 1, 2, -1, 2, True),
         (2, 2, 2, 1, 2, 1, 3, 1, 4, False)]


@functools.lru_cache(maxsize=None)
def _exact_joint(case):
    d, L, L_t, l, N, ns, nth, dirn, n, whole = case
    wv, F = ex.exact_path_measure(d, L, L_t, l, BETA, N, ns, nth, direction=dirn, n=n,
                                  whole=whole)
    dyn = ex._Dynamics(d, L, L_t, l, BETA, N, dirn, True, 1, n, whole)
    e_vals, e_idx = np.unique(dyn.energy(1.0).astype(np.int64), return_inverse=True)
    P = np.zeros((len(wv), len(e_vals)))
    for j in range(len(e_vals)):
        P[:, j] = F[:, e_idx == j].sum(axis=1)
    return wv, P, e_idx


def joint_law_pvalue(case, n_traj, lib=None, seed=4):
    d, L, L_t, l, N, ns, nth, dirn, n, whole = case
    wv, P, e_idx = _exact_joint(case)
    W, S = oracle.run(d, L, L_t, BETA, l, N, ns, n_traj, seed, n_therm=nth, direction=dirn,
                      want_spins=True, lib=lib, n_replica=n, whole=whole)
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
def test_law_matches_exact_path_measure(case):
    p, stray, stray_expected = joint_law_pvalue(case, 100_000)
    assert p > 1e-4
    assert stray <= stray_expected + 6 * math.sqrt(stray_expected + 1)


@pytest.mark.parametrize("mutant", [3, 6])
def test_planted_mistakes_are_caught(mutant, tmp_path):
    lib = oracle.load_library(oracle.build(out=str(tmp_path / f"liboracle_m{mutant}.so"),
                                           mutant=mutant))
    worst = 1.0
    for case in CASES[:3]:
        p, stray, stray_expected = joint_law_pvalue(case, 100_000, lib=lib)
        if stray > stray_expected + 6 * math.sqrt(stray_expected + 1):
            p = 0.0
        worst = min(worst, p)
    assert worst < 1e-8


@pytest.mark.parametrize("update", [0, 1])
def test_delta_s3_agrees_with_transfer_matrix(update):
    d, L, L_t, l, N, n = 2, 4, 8, 1, 20, 3
    exact = ex.delta_sn_transfer(d, L, L_t, BETA, n)[l]
    W, _ = oracle.run(d, L, L_t, BETA, l, N, 1, 4000, 31, n_therm=100, update=update,
                      n_replica=n)
    val, err = est.delta_s2_with_error(W, BETA, N)
    val, err = val / (n - 1), err / (n - 1)
    assert abs(val - exact) < 4 * err + 1e-3 * abs(exact)


@pytest.mark.parametrize("update", [0, 1])
@pytest.mark.parametrize("n", [2, 3])
def test_whole_cut_entropy_agrees_with_transfer_matrix(update, n):
    d, L, L_t, l, N = 2, 4, 8, 2, 40
    exact = ex.renyi_sn_transfer(d, L, L_t, BETA, n)[l]
    W, _ = oracle.run(d, L, L_t, BETA, l, N, 1, 4000, 33, n_therm=100, update=update,
                      n_replica=n, whole=True)
    val, err = est.delta_s2_with_error(W, BETA, N)
    val, err = val / (n - 1), err / (n - 1)
    assert abs(val - exact) < 4 * err + 1e-3 * abs(exact)


def test_bad_replica_arguments():
    for kw in (dict(n_replica=1), dict(whole=True, l=0), dict(whole=True, protocol=2),
               dict(n_replica=17)):
        args = dict(d=2, L=4, L_t=4, beta=BETA, l=1, n_step=4, n_sweep=1, n_traj=2, seed=0)
        extra = {k: v for k, v in kw.items() if k not in args}
        args.update({k: v for k, v in kw.items() if k in args})
        with pytest.raises(ValueError):
            oracle.run(*args.values(), n_therm=1, **extra)
