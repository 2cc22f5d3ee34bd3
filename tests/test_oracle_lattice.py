"""Pins of the oracle's D2Q9 / MRT algebra against exact rational arithmetic (Sec. II B, Eqs. 42-44, 53)."""

from fractions import Fraction

import numpy as np

from oracle import lattice as L
from oracle import model


def _mat_fr():
    return [[Fraction(int(v)) for v in row] for row in L.M_INT]


def test_weights_and_velocities():
    # Sec. II B: w0 = 4/9, w1-4 = 1/9, w5-8 = 1/36; isotropy sum w e_i e_j = c_s^2 delta_ij
    assert sum(L.W_FRAC) == 1
    assert L.W_FRAC[0] == Fraction(4, 9) and L.W_FRAC[1] == Fraction(1, 9) and L.W_FRAC[5] == Fraction(1, 36)
    for i, ei in enumerate((L.EX, L.EY)):
        for j, ej in enumerate((L.EX, L.EY)):
            s = sum(L.W_FRAC[a] * int(ei[a]) * int(ej[a]) for a in range(9))
            assert s == (Fraction(1, 3) if i == j else 0)
    for a in range(9):
        assert L.EX[L.OPP[a]] == -L.EX[a] and L.EY[L.OPP[a]] == -L.EY[a]


def test_m_inverse_exact():
    Mf = _mat_fr()
    Mi = L.m_inverse_fractions()
    for i in range(9):
        for j in range(9):
            assert sum(Mi[i][k] * Mf[k][j] for k in range(9)) == (1 if i == j else 0)
    assert np.allclose(L.MINV @ L.M, np.eye(9), atol=1e-15)


def test_eq44_is_moments_of_eq29():
    """Eq. 44 states m_eq = T(1,-2,1,vx,-vx,vy,-vy,0,0) is M applied to g_eq of Eq. 29,
    g_eq = w T (1 + e.v / c_s^2). This pins the row order and signs of M and the velocity order."""
    Mf = _mat_fr()
    for T, vx, vy in [(Fraction(3, 7), Fraction(1, 11), Fraction(-2, 13)), (Fraction(5), Fraction(-1, 3), Fraction(1, 5))]:
        geq = [L.W_FRAC[a] * T * (1 + 3 * (int(L.EX[a]) * vx + int(L.EY[a]) * vy)) for a in range(9)]
        m = [sum(Mf[k][a] * geq[a] for a in range(9)) for k in range(9)]
        assert m == [T, -2 * T, T, T * vx, -T * vx, T * vy, -T * vy, 0, 0]


def test_heat_equilibria_moments():
    """Both thermal equilibria (Eq. 44 and Eq. 53) have zeroth moment T, first moment T v and
    isotropic second moment c_s^2 T (the flux the Chapman-Enskog analysis, Eqs. A8-A9, relies on);
    Eq. 53 in addition has m1 + m2 = 0 (text after Eq. 52)."""
    rng = np.random.default_rng(0)
    T = rng.uniform(0.05, 0.2, (3, 4))
    vx = rng.uniform(-0.1, 0.1, (3, 4))
    vy = rng.uniform(-0.1, 0.1, (3, 4))
    for mdl in ("improved", "compromised"):
        meq = model.heat_meq(T, vx, vy, mdl)
        g = L.from_moments(meq)
        assert np.allclose(g.sum(0), T, rtol=1e-14)
        assert np.allclose(np.tensordot(L.EX.astype(float), g, 1), T * vx, atol=1e-15)
        assert np.allclose(np.tensordot(L.EY.astype(float), g, 1), T * vy, atol=1e-15)
        exx = np.tensordot((L.EX * L.EX).astype(float), g, 1)
        eyy = np.tensordot((L.EY * L.EY).astype(float), g, 1)
        exy = np.tensordot((L.EX * L.EY).astype(float), g, 1)
        assert np.allclose(exx, T / 3, rtol=1e-14) and np.allclose(eyy, T / 3, rtol=1e-14)
        assert np.allclose(exy, 0, atol=1e-16)
    meq = model.heat_meq(T, vx, vy, "improved")
    assert np.allclose(meq[1] + meq[2], 0)


def test_flow_equilibrium_is_second_order_maxwellian():
    """The flow m_eq maps back to the standard second-order D2Q9 equilibrium
    w rho (1 + 3 e.v + 4.5 (e.v)^2 - 1.5 v^2) (a textbook closed form)."""
    rng = np.random.default_rng(1)
    rho = rng.uniform(0.3, 6.5, (2, 3))
    vx = rng.uniform(-0.1, 0.1, (2, 3))
    vy = rng.uniform(-0.1, 0.1, (2, 3))
    f = L.from_moments(model.flow_meq(rho, vx, vy))
    for a in range(9):
        ev = L.EX[a] * vx + L.EY[a] * vy
        ref = L.W[a] * rho * (1 + 3 * ev + 4.5 * ev * ev - 1.5 * (vx * vx + vy * vy))
        assert np.allclose(f[a], ref, rtol=1e-13)
