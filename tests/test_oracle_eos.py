"""Pins of the oracle's Peng-Robinson EOS (Eq. 56) against closed forms and textbook facts."""

import math

import numpy as np
import pytest
from scipy import integrate, optimize

from oracle import eos

A, B, R, OM = 3.0 / 49.0, 2.0 / 21.0, 1.0, 0.344
TC = eos.critical_temperature(A, B, R)


def test_critical_point_is_inflection():
    """At T_c the isotherm has a horizontal inflection; for Peng-Robinson b rho_c = 0.25307 and
    Z_c = p_c/(rho_c R T_c) = 0.3074 (textbook values of the cubic). The constants 0.45724 and
    0.0778 of Eq. 56 are rounded, so the pin is to ~1e-4."""
    r = np.linspace(1.0, 4.0, 300001)
    d = eos.dp_drho(r, TC, A, B, R, OM)
    i = int(np.argmin(d))
    assert abs(d[i]) < 1e-3 * R * TC
    assert abs(B * r[i] - 0.25307) < 2e-4
    pc = eos.pressure(r[i], TC, A, B, R, OM)
    assert abs(pc / (r[i] * R * TC) - 0.3074) < 5e-4
    assert abs(pc - eos.critical_pressure(A, B, R)) / pc < 1e-3
    assert eos.theta(TC, TC, OM) == 1.0


def test_derivatives_match_finite_differences():
    rho = np.array([0.2, 0.38, 1.0, 2.657, 5.0, 6.5, 8.0])
    for T in (0.8 * TC, 0.86 * TC, TC, 1.25 * TC):
        h = 1e-6 * T
        fd = (eos.pressure(rho, T + h, A, B, R, OM) - eos.pressure(rho, T - h, A, B, R, OM)) / (2 * h)
        assert np.allclose(eos.dp_dT(rho, T, A, B, R, OM), fd, rtol=1e-7, atol=1e-10)
        hr = 1e-6 * rho
        fr = (eos.pressure(rho + hr, T, A, B, R, OM) - eos.pressure(rho - hr, T, A, B, R, OM)) / (2 * hr)
        assert np.allclose(eos.dp_drho(rho, T, A, B, R, OM), fr, rtol=1e-6, atol=1e-9)


def test_ideal_gas_limit():
    for T in (0.5 * TC, TC, 2 * TC):
        rho = 1e-7
        assert abs(eos.pressure(rho, T, A, B, R, OM) / (rho * R * T) - 1) < 1e-5


def _ln_fugacity_coeff(Z, Aa, Bb):
    """Textbook Peng-Robinson fugacity coefficient of a pure fluid."""
    s2 = math.sqrt(2.0)
    return (Z - 1) - math.log(Z - Bb) - Aa / (2 * s2 * Bb) * math.log((Z + (1 + s2) * Bb) / (Z + (1 - s2) * Bb))


@pytest.mark.parametrize("ratio", [0.7, 0.8, 0.86, 0.9, 0.95])
def test_maxwell_equal_fugacity(ratio):
    """Coexistence = equal pressure and equal fugacity (closed form, independent of the equal-area
    quadrature the oracle uses)."""
    T = ratio * TC
    rv, rl, ps = eos.maxwell_coexistence(T, A, B, R, OM)
    assert rv < rl
    pv, pl = eos.pressure(rv, T, A, B, R, OM), eos.pressure(rl, T, A, B, R, OM)
    assert abs(pv - ps) < 1e-12 * max(1.0, ps) and abs(pl - ps) < 1e-11 * max(1.0, ps)
    aT = A * eos.theta(T, TC, OM)
    Aa = aT * ps / (R * T) ** 2
    Bb = B * ps / (R * T)
    lv = _ln_fugacity_coeff(ps / (rv * R * T), Aa, Bb)
    ll = _ln_fugacity_coeff(ps / (rl * R * T), Aa, Bb)
    assert abs(lv - ll) < 1e-9


def test_maxwell_equal_area_scipy():
    """The equal-area integral, re-done with scipy's adaptive quadrature, vanishes."""
    T = 0.86 * TC
    rv, rl, ps = eos.maxwell_coexistence(T, A, B, R, OM)
    val, _ = integrate.quad(lambda r: (eos.pressure(r, T, A, B, R, OM) - ps) / r ** 2, rv, rl, limit=200, epsabs=1e-14)
    scale, _ = integrate.quad(lambda r: abs(eos.pressure(r, T, A, B, R, OM) - ps) / r ** 2, rv, rl, limit=200)
    assert abs(val) < 1e-10 * scale
    # coexistence densities of the paper's working point (T_sat = 0.86 T_c): density ratio about 17
    assert 16.5 < rl / rv < 17.5


def test_psi_real_at_working_point():
    """psi^2 = 2 (p_EOS - rho/3)/G must be positive over the liquid-vapour range near T_sat and in
    hot vapour up to the heated-wall temperature 1.25 T_c (Sec. IV B); it turns negative for dense,
    hot fluid, which the step reports as a non-physical state."""
    for T, top in ((0.80 * TC, 7.5), (0.86 * TC, 7.5), (0.95 * TC, 7.0), (1.16 * TC, 2.0), (1.25 * TC, 2.0)):
        rho = np.linspace(0.05, top, 400)
        p = eos.pressure(rho, T, A, B, R, OM)
        assert np.all(eos.psi_squared(rho, p, -1.0) > 0)
    p = eos.pressure(8.0, 1.25 * TC, A, B, R, OM)
    assert eos.psi_squared(8.0, p, -1.0) < 0
