"""FP64 estimator of the oracle: Jarzynski average, Renyi-2 increment, jackknife,
entropic c-function.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* ``log_mean_exp_neg``  ln <exp(-W)> over trajectories (Appendix A, eq.
  Jarzynski_theorem), with W = beta W_int / N, written as a max-shifted sum.
* ``delta_s2``          Delta S_2(l -> l+1) = -ln[Z_2(l+1)/Z_2(l)]
  (section 2, eqs. trace_of_rho_n_as_ratio_of_partition_functions and
  definition_of_derivative_of_Renyi_entropy with n = 2, epsilon = a = 1).
* ``jackknife``         blocked jackknife over contiguous trajectory blocks.
* ``c_function``        symmetrised entropic c-function (section 2, eq.
  symmetrised_entropic_c-function) at the midpoint x = (l + 1/2)/L of the
  finite difference (Appendix C).
* ``entropy_increments`` the increment trick (section 3): S_2(l) up to a
  constant as the running sum of Delta S_2.
"""
from __future__ import annotations

import math

import numpy as np


def work_values(work_int, beta: float, n_step: int) -> np.ndarray:
    """W_i = beta * W_int_i / N (the work of Appendix A in units of T)."""
    return beta * np.asarray(work_int, dtype=np.float64) / float(n_step)


def log_mean_exp_neg(w) -> float:
    """ln( (1/n) sum_i exp(-w_i) ) computed as m + ln sum exp(-w_i - m) - ln n,
    m = max_i(-w_i)."""
    w = np.asarray(w, dtype=np.float64)
    if w.size == 0:
        raise ValueError("empty work sample")
    neg = -w
    m = float(np.max(neg))
    return m + math.log(float(np.sum(np.exp(neg - m)))) - math.log(w.size)


def delta_s2(work_int, beta: float, n_step: int, direction: int = 1) -> float:
    """Delta S_2(l -> l+1).  Forward runs estimate <e^-W> = Z_2(l+1)/Z_2(l), so
    Delta S_2 = -ln<e^-W>; reverse runs estimate its inverse (Appendix A, eq.
    equality_of_direct_reverse_protocols), so Delta S_2 = +ln<e^-W>."""
    lme = log_mean_exp_neg(work_values(work_int, beta, n_step))
    return -lme if direction > 0 else lme


def jackknife_blocks(n: int, n_blocks: int = 32):
    """B = min(n_blocks, n) contiguous blocks of size n // B; the remainder
    joins the last block.  Returns a list of (start, stop)."""
    B = min(n_blocks, n)
    size = n // B
    edges = [b * size for b in range(B)] + [n]
    return [(edges[b], edges[b + 1]) for b in range(B)]


def jackknife(values, estimator, n_blocks: int = 32):
    """(estimate on all data, blocked-jackknife error).

    theta_b = estimator(values without block b); error =
    sqrt((B-1)/B * sum_b (theta_b - mean_b theta_b)^2)."""
    values = np.asarray(values)
    full = estimator(values)
    blocks = jackknife_blocks(len(values), n_blocks)
    B = len(blocks)
    if B < 2:
        return full, float("nan")
    thetas = np.array([estimator(np.concatenate([values[:a], values[b:]]))
                       for a, b in blocks])
    err = math.sqrt((B - 1) / B * float(np.sum((thetas - thetas.mean()) ** 2)))
    return full, err


def delta_s2_with_error(work_int, beta, n_step, direction=1, n_blocks=32):
    est = lambda wi: delta_s2(wi, beta, n_step, direction)
    return jackknife(np.asarray(work_int, dtype=np.int64), est, n_blocks)


def c_function(ds2, d: int, L: int, l: int) -> float:
    """C_2 at x = (l + 1/2)/L from Delta S_2(l -> l+1):
    [(L/pi) sin(pi x)]^(d-1) / |dA| * dS_2/dl with |dA| = 2 L^(d-2) (two
    boundary points in 2D, two lines of length L in 3D) and dS_2/dl ~ Delta S_2."""
    x = (l + 0.5) / L
    arc = (L / math.pi) * math.sin(math.pi * x)
    return arc ** (d - 1) * ds2 / (2.0 * L ** (d - 2))


def entropy_increments(ds2_values) -> np.ndarray:
    """S_2(l) - S_2(l_0) for l = l_0, l_0+1, ..., as the running sum of
    Delta S_2 (the increment trick of section 3)."""
    return np.concatenate([[0.0], np.cumsum(np.asarray(ds2_values, dtype=np.float64))])


def cft_delta_s2(L: int, l: int, c: float = 0.5, n: int = 2) -> float:
    """Delta S_n between l and l+1 from the cylinder CFT form
    S_n = (c/6)(1 + 1/n) ln[(L/pi) sin(pi l/L)] + k_n (section 2)."""
    pref = c / 6.0 * (1.0 + 1.0 / n)
    return pref * math.log(math.sin(math.pi * (l + 1) / L) / math.sin(math.pi * l / L))
