"""Peng-Robinson equation of state and the pseudopotential it feeds (oracle; test infrastructure only).

Eq. 56:  p_EOS = rho R T / (1 - b rho) - a theta(T) rho^2 / (1 + 2 b rho - b^2 rho^2),
         theta(T) = [1 + kappa (1 - sqrt(T/T_c))]^2,
         kappa = 0.37464 + 1.54226 omega - 0.26992 omega^2,
         a = 0.45724 R^2 T_c^2 / p_c,  b = 0.0778 R T_c / p_c,
with a = 3/49, b = 2/21, R = 1, omega = 0.344 and T_sat = 0.86 T_c (text after Eq. 56).
T_c "can be obtained from the formulations of a and b": dividing the two gives
T_c = 0.0778 a / (0.45724 b R), and then p_c = 0.0778 R T_c / b.

(dp/dT)_rho (needed by the source term of Eqs. 5, 13 and 28) is the analytic T-derivative of Eq. 56.

READING (the paper follows Ref. [48] and Refs. [13,29] for the flow model without restating the
mapping): the pseudopotential is psi = sqrt(2 (p_EOS - rho c_s^2) / (G c^2)) with G = -1, the
standard EOS-to-psi mapping of the pseudopotential method.
"""

import math

import numpy as np

CS2 = 1.0 / 3.0


def kappa(omega):
    """kappa(omega) of theta(T) in Eq. 56."""
    return 0.37464 + 1.54226 * omega - 0.26992 * omega * omega


def critical_temperature(a, b, R):
    """T_c from a = 0.45724 R^2 T_c^2/p_c and b = 0.0778 R T_c/p_c (text after Eq. 56)."""
    return 0.0778 * a / (0.45724 * b * R)


def critical_pressure(a, b, R):
    """p_c = 0.0778 R T_c / b (text after Eq. 56)."""
    return 0.0778 * R * critical_temperature(a, b, R) / b


def theta(T, Tc, omega):
    """theta(T) = [1 + kappa (1 - sqrt(T/T_c))]^2 (Eq. 56)."""
    return (1.0 + kappa(omega) * (1.0 - np.sqrt(T / Tc))) ** 2


def dtheta_dT(T, Tc, omega):
    """d theta / dT = -kappa [1 + kappa (1 - sqrt(T/T_c))] / sqrt(T T_c) (derivative of Eq. 56's theta)."""
    k = kappa(omega)
    return -k * (1.0 + k * (1.0 - np.sqrt(T / Tc))) / np.sqrt(T * Tc)


def pressure(rho, T, a, b, R, omega):
    """p_EOS(rho, T), Eq. 56."""
    Tc = critical_temperature(a, b, R)
    return rho * R * T / (1.0 - b * rho) - a * theta(T, Tc, omega) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho)


def dp_dT(rho, T, a, b, R, omega):
    """(dp_EOS/dT)_rho, the T-derivative of Eq. 56 at fixed rho."""
    Tc = critical_temperature(a, b, R)
    return rho * R / (1.0 - b * rho) - a * dtheta_dT(T, Tc, omega) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho)


def dp_drho(rho, T, a, b, R, omega):
    """(dp_EOS/drho)_T = R T/(1-b rho)^2 - a theta 2 rho (1 + b rho)/(1 + 2 b rho - b^2 rho^2)^2."""
    Tc = critical_temperature(a, b, R)
    d = 1.0 + 2.0 * b * rho - b * b * rho * rho
    return R * T / (1.0 - b * rho) ** 2 - a * theta(T, Tc, omega) * 2.0 * rho * (1.0 + b * rho) / (d * d)


def psi_squared(rho, p, G):
    """psi^2 = 2 (p_EOS - rho c_s^2) / (G c^2), c = 1 (READING of the delegated flow model)."""
    return 2.0 * (p - rho * CS2) / G


def _bisect(fun, lo, hi, iters=200):
    flo = fun(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = fun(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
        if hi - lo <= 1e-15 * max(1.0, abs(lo)):
            break
    return 0.5 * (lo + hi)


def spinodals(T, a, b, R, omega, n_scan=20000):
    """The two roots of (dp/drho)_T = 0 below T_c, found by a scan for sign changes then bisection."""
    rmax = 1.0 / b
    grid = np.linspace(rmax * 1e-6, rmax * (1 - 1e-6), n_scan)
    d = dp_drho(grid, T, a, b, R, omega)
    idx = np.nonzero(np.sign(d[1:]) != np.sign(d[:-1]))[0]
    if len(idx) != 2:
        raise ValueError("no two spinodals: T is not below T_c")
    f = lambda r: dp_drho(r, T, a, b, R, omega)  # noqa: E731
    return tuple(_bisect(f, grid[i], grid[i + 1]) for i in idx)


def _gauss_legendre_integral(fun, lo, hi, panels=400, order=8):
    x, w = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(lo, hi, panels + 1)
    total = 0.0
    for k in range(panels):
        l, h = edges[k], edges[k + 1]
        xs = 0.5 * (h - l) * x + 0.5 * (h + l)
        total += 0.5 * (h - l) * float(np.dot(w, fun(xs)))
    return total


def maxwell_coexistence(T, a, b, R, omega):
    """Coexistence densities (rho_v, rho_l) and p_sat at temperature T by Maxwell's equal-area rule.

    At coexistence p(rho_v) = p(rho_l) = p_s and the loop of p against specific volume V = 1/rho
    encloses equal areas: int_{rho_v}^{rho_l} (p(rho) - p_s) / rho^2 drho = 0. The paper sets the
    saturation temperature T_sat = 0.86 T_c (after Eq. 56); the densities follow from Eq. 56.
    Bisection on p_s between the spinodal pressures; the outer roots by bisection; the area by
    composite Gauss-Legendre quadrature in u = ln rho.
    """
    r1, r2 = spinodals(T, a, b, R, omega)
    p = lambda r: pressure(r, T, a, b, R, omega)  # noqa: E731
    p_lo, p_hi = max(p(r2), 1e-300), p(r1)
    rmax = 1.0 / b

    def roots(ps):
        # p ~ rho R T as rho -> 0, so p(rho) < p_s at rho = p_s / (2 R T): a valid lower bracket
        rv = _bisect(lambda r: p(r) - ps, min(1e-12, 0.5 * ps / (R * T)), r1)
        rl = _bisect(lambda r: p(r) - ps, r2, rmax * (1.0 - 1e-12))
        return rv, rl

    def area(ps):
        # substitute rho = exp(u): the integrand (p - p_s)/rho stays bounded as rho_v -> 0
        rv, rl = roots(ps)
        return _gauss_legendre_integral(lambda u: (p(np.exp(u)) - ps) / np.exp(u), math.log(rv), math.log(rl))

    ps = _bisect(area, p_lo + 1e-14 * abs(p_hi), p_hi - 1e-14 * abs(p_hi), iters=200)
    rv, rl = roots(ps)
    return rv, rl, ps
