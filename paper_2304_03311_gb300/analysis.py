"""Analysis of Renyi-entropy increments and entropic c-functions (host side).

What a user does with the Delta S_n values the library estimates:

* the symmetrised entropic c-function at the midpoint of each l -> l+1 move
  (section 2, eq. symmetrised_entropic_c-function);
* the Renyi entropy itself by summing increments (the increment trick,
  section 3);
* the 2D fit with the leading finite-size correction (section 4, eq.
  fit_function_2d) and the comparison with the scaling function alone;
* the three 3D families for S_2 and their c-functions (section 5, eqs.
  fit_entropy_2d_analogue_3d, fit_entropy_RVB_3d, fit_entropy_AdS_3d and
  fit_c-fun_*_3d), fitted by weighted least squares;
* the systematic error of the finite difference (Appendix C, eq.
  entropic_c-function_and_third_derivative);
* the Kramers-Wannier dual coupling (section 4, "Variation with beta").

Pure numpy / scipy; nothing here touches the GPU.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy import integrate, optimize

BETA_C_2D = 0.5 * math.log(1.0 + math.sqrt(2.0))


# --------------------------------------------------------------- c-function --
def midpoint_x(l, L):
    """x = (l + 1/2)/L, where the l -> l+1 finite difference is centred."""
    return (np.asarray(l, dtype=float) + 0.5) / float(L)


def c_function(delta_s, d: int, L: int, l, err=None):
    """Symmetrised entropic c-function from Delta S_n(l -> l+1):
    C_n(x) = [(L/pi) sin(pi x)]^(d-1) Delta S_n / (2 L^(d-2)) at x = (l+1/2)/L
    (the area |dA| of the entangling surface is 2 L^(d-2) on the torus).
    Returns C, or (C, error) when err is given."""
    x = midpoint_x(l, L)
    factor = (L / math.pi * np.sin(math.pi * x)) ** (d - 1) / (2.0 * L ** (d - 2))
    c = factor * np.asarray(delta_s, dtype=float)
    if err is None:
        return c
    return c, factor * np.asarray(err, dtype=float)


def renyi_from_increments(delta_s, err=None):
    """S_n(l) for l = 0..len: S_n(0) = 0 and S_n(l+1) = S_n(l) + Delta S_n(l)
    (the increment trick).  Independent increments: errors add in quadrature."""
    s = np.concatenate([[0.0], np.cumsum(np.asarray(delta_s, dtype=float))])
    if err is None:
        return s
    e = np.concatenate([[0.0], np.sqrt(np.cumsum(np.asarray(err, dtype=float) ** 2))])
    return s, e


# ------------------------------------------------------------- weighted fits --
@dataclass
class Fit:
    params: np.ndarray      # best-fit parameters
    errors: np.ndarray      # their standard errors
    chi2: float
    dof: int

    @property
    def chi2_per_dof(self) -> float:
        return self.chi2 / self.dof if self.dof > 0 else float("nan")


def _linear_fit(basis: np.ndarray, y, err) -> Fit:
    """Weighted least squares y ~ basis @ p with standard errors err."""
    y = np.asarray(y, dtype=float)
    w = 1.0 / np.asarray(err, dtype=float)
    A = basis * w[:, None]
    b = y * w
    p, *_ = np.linalg.lstsq(A, b, rcond=None)
    cov = np.linalg.inv(A.T @ A)
    r = A @ p - b
    return Fit(p, np.sqrt(np.diag(cov)), float(r @ r), len(y) - basis.shape[1])


def _trim(drop_ends: int, *arrays):
    if drop_ends <= 0:
        return arrays
    return tuple(np.asarray(a)[drop_ends:-drop_ends] for a in arrays)


def scaling_function_2d(x):
    """The 2D critical Ising c-function on the cylinder, cos(pi x)/16
    (section 4, eq. entropic_c-function_on_the_cylinder_2D with c = 1/2)."""
    return np.cos(math.pi * np.asarray(x, dtype=float)) / 16.0


def fit_function_2d(x, k: float, L: int):
    """f(x; k) = cos(pi x)/16 + k cot(pi x)/(2L) (section 4, eq. fit_function_2d)."""
    x = np.asarray(x, dtype=float)
    return scaling_function_2d(x) + k / (2.0 * L) / np.tan(math.pi * x)


def chi2_scaling_function_2d(x, c, err, drop_ends: int = 0) -> Fit:
    """chi^2 of the data against the scaling function alone (no free
    parameter); drop_ends removes that many points at each end."""
    x, c, err = _trim(drop_ends, x, c, err)
    r = (np.asarray(c) - scaling_function_2d(x)) / np.asarray(err)
    return Fit(np.zeros(0), np.zeros(0), float(r @ r), len(r))


def fit_2d(x, c, err, L: int, drop_ends: int = 0) -> Fit:
    """Best k of f(x; k) (linear in k): params = [k]."""
    x, c, err = _trim(drop_ends, x, c, err)
    x = np.asarray(x, dtype=float)
    y = np.asarray(c, dtype=float) - scaling_function_2d(x)
    basis = (1.0 / (2.0 * L) / np.tan(math.pi * x))[:, None]
    return _linear_fit(basis, y, err)


# ------------------------------------------------- theta and eta functions --
def theta3_imag(t: float) -> float:
    """Jacobi theta_3 at modular parameter tau = i t (t > 0):
    sum_n exp(-pi t n^2); for t < 1 through theta_3(i t) = t^(-1/2) theta_3(i/t)."""
    if t <= 0:
        raise ValueError("t must be positive")
    if t < 1.0:
        return theta3_imag(1.0 / t) / math.sqrt(t)
    q = math.exp(-math.pi * t)
    s, n = 1.0, 1
    while True:
        term = 2.0 * q ** (n * n)
        s += term
        if term < 1e-17 * s:
            return s
        n += 1


def eta_imag(t: float) -> float:
    """Dedekind eta at tau = i t (t > 0): exp(-pi t/12) prod_n (1 - exp(-2 pi n t));
    for t < 1 through eta(i t) = t^(-1/2) eta(i/t)."""
    if t <= 0:
        raise ValueError("t must be positive")
    if t < 1.0:
        return eta_imag(1.0 / t) / math.sqrt(t)
    q2 = math.exp(-2.0 * math.pi * t)
    p, n = 1.0, 1
    while True:
        f = q2 ** n
        p *= 1.0 - f
        if f < 1e-17:
            return math.exp(-math.pi * t / 12.0) * p
        n += 1


# ------------------------------------------------------------ 3D families --
def g_2d(x, c: float = 1.0, k: float = 0.0):
    """g_2D(x; c, k) = c log(sin(pi x)) + k (section 5, eq. fit_entropy_2d_analogue_3d)."""
    return c * np.log(np.sin(math.pi * np.asarray(x, dtype=float))) + k


def _rvb_shape(x: float, tau_imag: float) -> float:
    """-2 log{ eta(tau)^2/(theta3(2tau) theta3(tau/2)) *
    theta3(2x tau) theta3(2(1-x) tau)/(eta(2x tau) eta(2(1-x) tau)) } for tau = i tau_imag."""
    t = tau_imag
    pref = eta_imag(t) ** 2 / (theta3_imag(2 * t) * theta3_imag(t / 2))
    a, b = 2 * x * t, 2 * (1 - x) * t
    val = pref * theta3_imag(a) * theta3_imag(b) / (eta_imag(a) * eta_imag(b))
    return -2.0 * math.log(val)


def g_rvb(x, c: float = 1.0, k: float = 0.0, tau_imag: float = 1.0):
    """g_RVB(x; c, k) of the RVB dimer ground state (section 5, eq.
    fit_entropy_RVB_3d) with modular parameter tau = i tau_imag (tau = i on
    the L_y = L_x torus)."""
    xs = np.atleast_1d(np.asarray(x, dtype=float))
    out = np.array([_rvb_shape(float(v), tau_imag) for v in xs])
    out = c * out + k
    return out if np.ndim(x) else float(out[0])


def _ads_Q(chi: float, u: float) -> float:
    """P(chi, y)/u^2 at y = 1 - u^2, written without cancellation:
    1 - y^3 = u^2 (3 - 3u^2 + u^4) and 1 - y^4 = u^2 (4 - 6u^2 + 4u^4 - u^6)."""
    u2 = u * u
    return chi * (3.0 - 3.0 * u2 + u2 * u2) + (1.0 - chi) * (4.0 - 6.0 * u2 + 4.0 * u2 * u2
                                                            - u2 * u2 * u2)


def _ads_integrand_x(u, chi):
    # y = 1 - u^2 takes the 1/sqrt(P) endpoint singularity at y = 1 out
    u2 = u * u
    y = 1.0 - u2
    one_minus_chi_y3 = (1.0 - chi) + chi * u2 * (3.0 - 3.0 * u2 + u2 * u2)
    return 2.0 * y * y / (one_minus_chi_y3 * math.sqrt(_ads_Q(chi, u)))


def _ads_integrand_g(u, chi):
    # (1/sqrt(P) - 1)/y^2 = (chi y + (1 - chi) y^2)/(sqrt(P) (1 + sqrt(P)))
    y = 1.0 - u * u
    sq = math.sqrt(_ads_Q(chi, u))
    return 2.0 * (chi * y + (1.0 - chi) * y * y) / (sq * (1.0 + u * sq))


def ads_x_of_chi(chi: float) -> float:
    """x(chi) = 3/(2 pi) chi^(1/3) (1-chi)^(1/2) int_0^1 dy y^2 /((1 - chi y^3) sqrt(P))
    (section 5, below eq. fit_entropy_AdS_3d); rises from 0 at chi = 0 to 1/2
    at chi = 1."""
    peak = math.sqrt(max(1.0 - chi, 1e-300) / (3.0 * chi))
    pts = [peak] if 0.0 < peak < 1.0 else None
    val, _ = integrate.quad(_ads_integrand_x, 0.0, 1.0, args=(chi,), limit=400, points=pts,
                            epsabs=1e-14, epsrel=1e-12)
    return 1.5 / math.pi * chi ** (1.0 / 3.0) * math.sqrt(1.0 - chi) * val


def _ads_shape_of_chi(chi: float) -> float:
    val, _ = integrate.quad(_ads_integrand_g, 0.0, 1.0, args=(chi,), limit=400,
                            epsabs=1e-14, epsrel=1e-12)
    return chi ** (-1.0 / 3.0) * (val - 1.0)


def _chi_of_x(x: float) -> float:
    """Inverse of ads_x_of_chi for 0 < x <= 1/2 (x(chi) is increasing); within
    3e-7 of x = 1/2 the shape is flat to 1e-12 and chi = 1 - 1e-12 is used."""
    lo, hi = 1e-15, 1.0 - 1e-12
    if x >= ads_x_of_chi(hi):
        return hi
    return optimize.brentq(lambda c: ads_x_of_chi(c) - x, lo, hi, xtol=1e-15, rtol=1e-14,
                           maxiter=400)


def g_ads(x, c: float = 1.0, k: float = 0.0):
    """g_AdS(x; c, k) = c chi^(-1/3) { int_0^1 dy/y^2 (1/sqrt(P(chi,y)) - 1) - 1 } + k
    with chi = chi(x) (section 5, eq. fit_entropy_AdS_3d), symmetric about x = 1/2."""
    xs = np.atleast_1d(np.asarray(x, dtype=float))
    out = np.array([_ads_shape_of_chi(_chi_of_x(min(v, 1.0 - v))) for v in xs])
    out = c * out + k
    return out if np.ndim(x) else float(out[0])


FAMILIES = {"2d": g_2d, "rvb": g_rvb, "ads": g_ads}


def _derivative(g, x):
    """Central difference of order h^4 (five points), the step scaled to the
    distance from the singular ends x = 0, 1."""
    x = np.asarray(x, dtype=float)
    h = np.minimum(1e-4, np.minimum(x, 1.0 - x) / 100.0)
    return (-g(x + 2 * h) + 8 * g(x + h) - 8 * g(x - h) + g(x - 2 * h)) / (12.0 * h)


def c_function_family(family: str, x, c: float = 1.0):
    """The family's c-function f(x; c) = sin(pi x)^2/(2 pi^2) dg/dx (section 5,
    eqs. fit_c-fun_*_3d); for "2d" the closed form c sin(pi x) cos(pi x)/(2 pi)."""
    x = np.asarray(x, dtype=float)
    if family == "2d":
        return c / (2.0 * math.pi) * np.sin(math.pi * x) * np.cos(math.pi * x)
    g = FAMILIES[family]
    return c * np.sin(math.pi * x) ** 2 / (2.0 * math.pi ** 2) * _derivative(g, x)


def fit_entropy(family: str, x, s, err, drop_ends: int = 0) -> Fit:
    """Weighted least squares of S_2(x) = c shape(x) + k: params = [c, k]."""
    x, s, err = _trim(drop_ends, x, s, err)
    shape = np.asarray(FAMILIES[family](np.asarray(x, dtype=float)), dtype=float)
    basis = np.stack([shape, np.ones_like(shape)], axis=1)
    return _linear_fit(basis, s, err)


def fit_c_function(family: str, x, cf, err, drop_ends: int = 0) -> Fit:
    """Weighted least squares of C(x) = c f(x; 1): params = [c]."""
    x, cf, err = _trim(drop_ends, x, cf, err)
    basis = np.asarray(c_function_family(family, np.asarray(x, dtype=float)))[:, None]
    return _linear_fit(basis, cf, err)


# ------------------------------------------------ finite-difference systematics --
def third_derivative(g, x):
    """d^3 g/dx^3 by the central difference of order h^2, the step scaled to
    the distance from the singular ends x = 0, 1."""
    x = np.asarray(x, dtype=float)
    h = np.minimum(2e-3, np.minimum(x, 1.0 - x) / 40.0)
    return (g(x + 2 * h) - 2 * g(x + h) + 2 * g(x - h) - g(x - 2 * h)) / (2.0 * h ** 3)


def finite_difference_systematic(d: int, L: int, x, s_third):
    """C^MC(x) - C(x) = sin(pi x)^(D-1)/(48 L^2 pi^(D-1)) S'''(x) + O(1/L^4)
    (Appendix C, eq. entropic_c-function_and_third_derivative), S''' the third
    x-derivative of the Renyi entropy (from a fit, e.g. third_derivative of a
    fitted g)."""
    x = np.asarray(x, dtype=float)
    return np.sin(math.pi * x) ** (d - 1) / (48.0 * L ** 2 * math.pi ** (d - 1)) * \
        np.asarray(s_third, dtype=float)


# ------------------------------------------------------------ duality --
def kramers_wannier_dual(beta):
    """beta* with exp(-2 beta) = tanh(beta*) (section 4, Kramers and Wannier);
    an involution whose fixed point is beta_c = ln(1 + sqrt 2)/2."""
    return np.arctanh(np.exp(-2.0 * np.asarray(beta, dtype=float)))
