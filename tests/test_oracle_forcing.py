"""Pins of the oracle's flow collision with forcing (Sec. III B, closing paragraph: the flow model is
delegated to the paper's Refs. [13,29], the MRT pseudopotential model with its forcing scheme).

The MRT collision m* = m - Lambda (m - m_eq) + (I - Lambda/2) S_F reduces, when every rate in Lambda
is the same 1/tau, to the BGK collision with Guo's forcing term, a textbook closed form:

    f*_a = f_a - (f_a - f_a^eq(rho, v)) / tau
           + (1 - 1/(2 tau)) w_a [ (e_a - v) / c_s^2 + (e_a . v) e_a / c_s^4 ] . F,
    f_a^eq = w_a rho [1 + e_a.v / c_s^2 + (e_a.v)^2 / (2 c_s^4) - v^2 / (2 c_s^2)].

That statement is written out below from its own D2Q9 table, independent of oracle.lattice, and the
oracle's collision is checked against it node by node. Random v and F with both components nonzero
make every row of S_F matter: the 6 v.F of the energy moments, the force rows and the two
velocity-dependent stress rows 2 (vx Fx - vy Fy) and vx Fy + vy Fx.

The sigma term Q = 12 sigma |F_int|^2 / (psi^2 (1/s_e - 1/2)) of the mechanical-stability correction
enters the energy moments only: m1* gains (1 - s_e/2) Q and m2* loses (1 - s_eps/2) Q. Its check builds
F_int from a psi field in closed form (a sine mode along x, for which the interaction sum is exact).
"""

import numpy as np
import pytest

from oracle import model

# D2Q9, written out here (same velocity order as the paper's Sec. II B)
E = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)], dtype=float)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0


def _bgk_guo(f, rho, vx, vy, Fx, Fy, tau):
    out = np.empty_like(f)
    v2 = vx * vx + vy * vy
    for a in range(9):
        ex, ey = E[a]
        ev = ex * vx + ey * vy
        eF = ex * Fx + ey * Fy
        feq = W[a] * rho * (1 + ev / CS2 + ev * ev / (2 * CS2 * CS2) - v2 / (2 * CS2))
        guo = W[a] * (((ex - vx) * Fx + (ey - vy) * Fy) / CS2 + ev * eF / (CS2 * CS2))
        out[a] = f[a] - (f[a] - feq) / tau + (1 - 1 / (2 * tau)) * guo
    return out


def _inputs(seed, shape=(6, 7)):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.4, 6.5, shape)
    vx, vy = rng.uniform(-0.08, 0.08, shape), rng.uniform(-0.08, 0.08, shape)
    Fx, Fy = rng.uniform(-0.02, 0.02, shape), rng.uniform(-0.02, 0.02, shape)
    # populations near equilibrium, perturbed in every direction (so every moment is off equilibrium)
    f = np.stack([W[a] * rho * (1 + 0.2 * rng.uniform(-1, 1, shape)) for a in range(9)])
    return f, rho, vx, vy, Fx, Fy


def _mac(rho, vx, vy, Fx, Fy, Fix=None, Fiy=None, psi=None):
    z = np.zeros_like(rho)
    return dict(rho=rho, vx=vx, vy=vy, Fx=Fx, Fy=Fy, Fix=z if Fix is None else Fix, Fiy=z if Fiy is None else Fiy,
                psi=np.ones_like(rho) if psi is None else psi)


@pytest.mark.parametrize("tau", [0.8, 1.37])
def test_equal_rates_reduce_to_bgk_with_guo_forcing(tau):
    f, rho, vx, vy, Fx, Fy = _inputs(int(tau * 100))
    p = model.OracleParams(nx=7, ny=6, s_f=(1.0 / tau,) * 9, sigma=0.0)
    got = model.collide_flow(p, f, _mac(rho, vx, vy, Fx, Fy))
    ref = _bgk_guo(f, rho, vx, vy, Fx, Fy, tau)
    assert np.max(np.abs(got - ref)) < 1e-14 * np.max(np.abs(ref))
    # each kind of term contributes well above that tolerance: the forcing, and in it the v-dependent part
    assert np.max(np.abs(_bgk_guo(f, rho, vx, vy, Fx, Fy, tau) - _bgk_guo(f, rho, vx, vy, 0 * Fx, 0 * Fy, tau))) > 1e-4
    vdep = _bgk_guo(f, rho, vx, vy, Fx, Fy, tau) - _bgk_guo(f, rho, vx, vy, 0 * Fx, 0 * Fy, tau)
    vfree = _bgk_guo(f, rho, 0 * vx, 0 * vy, Fx, Fy, tau) - _bgk_guo(f, rho, 0 * vx, 0 * vy, 0 * Fx, 0 * Fy, tau)
    assert np.max(np.abs(vdep - vfree)) > 1e-5


def test_collision_conserves_mass_and_adds_the_force():
    """For any rates: sum f* = rho and sum e f* = j + F when v = (j + F/2)/rho (the forcing scheme's
    velocity), i.e. the conserved moments do not depend on their rates."""
    f, rho, _, _, Fx, Fy = _inputs(7)
    jx = (E[:, 0, None, None] * f).sum(0)
    jy = (E[:, 1, None, None] * f).sum(0)
    rho = f.sum(0)
    vx, vy = (jx + Fx / 2) / rho, (jy + Fy / 2) / rho
    p = model.OracleParams(nx=7, ny=6, s_f=(0.6, 0.8, 0.9, 1.3, 1.1, 0.7, 1.1, 1.25, 1.25), sigma=0.0)
    fs = model.collide_flow(p, f, _mac(rho, vx, vy, Fx, Fy))
    assert np.allclose(fs.sum(0), rho, rtol=1e-14)
    assert np.allclose((E[:, 0, None, None] * fs).sum(0), jx + Fx, atol=1e-14)
    assert np.allclose((E[:, 1, None, None] * fs).sum(0), jy + Fy, atol=1e-14)


def test_sigma_term_enters_only_the_energy_moments():
    """Q = 12 sigma |F_int|^2 / (psi^2 (1/s_e - 1/2)): with everything else fixed, sigma changes the
    post-collision energy moment e by +(1 - s_e/2) Q and eps by -(1 - s_eps/2) Q, and nothing else.

    F_int comes from psi = psi0 + eps sin(q x) in closed form: with G = -1 and the interaction
    weights 1/3 (axes) and 1/12 (diagonals), sum_a w psi(x + e_a) e_ax = (1/3 + 2/12)(psi(x+1) - psi(x-1))
    = eps sin(q) cos(q x), so F_int,x = psi eps sin(q) cos(q x) and F_int,y = 0."""
    nx, ny = 16, 3
    q = 2 * np.pi / nx
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    psi0, eps = 1.1, 0.05
    psi = psi0 + eps * np.sin(q * x)
    Fix = psi * eps * np.sin(q) * np.cos(q * x)
    Fiy = np.zeros_like(psi)
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.4, 6.5, psi.shape)
    vx, vy = rng.uniform(-0.05, 0.05, psi.shape), rng.uniform(-0.05, 0.05, psi.shape)
    f = np.stack([W[a] * rho * (1 + 0.1 * rng.uniform(-1, 1, psi.shape)) for a in range(9)])
    s_f = (1.0, 0.8, 0.7, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25)
    mac = _mac(rho, vx, vy, Fix, Fiy, Fix, Fiy, psi)
    sigma = 0.1
    f0 = model.collide_flow(model.OracleParams(nx=nx, ny=ny, s_f=s_f, sigma=0.0), f, mac)
    f1 = model.collide_flow(model.OracleParams(nx=nx, ny=ny, s_f=s_f, sigma=sigma), f, mac)
    d = f1 - f0
    # moments of the difference, by the D2Q9 polynomials of the two energy moments
    e2 = (E ** 2).sum(1)
    m_e = ((3 * e2 - 4)[:, None, None] * d).sum(0)
    m_eps = ((4.5 * e2 * e2 - 10.5 * e2 + 4)[:, None, None] * d).sum(0)
    Q = 12 * sigma * (Fix ** 2 + Fiy ** 2) / (psi ** 2 * (1 / s_f[1] - 0.5))
    assert np.max(Q) > 1e-5
    assert np.allclose(m_e, (1 - s_f[1] / 2) * Q, rtol=1e-9, atol=1e-13 * np.max(np.abs(f)))
    assert np.allclose(m_eps, -(1 - s_f[2] / 2) * Q, rtol=1e-9, atol=1e-13 * np.max(np.abs(f)))
    # every other moment (mass, momentum, heat fluxes, stresses) is unchanged, up to the rounding of f
    tol = 1e-14 * np.max(np.abs(f))
    others = [np.ones(9), E[:, 0], E[:, 1], (3 * e2 - 5) * E[:, 0], (3 * e2 - 5) * E[:, 1],
              E[:, 0] ** 2 - E[:, 1] ** 2, E[:, 0] * E[:, 1]]
    for poly in others:
        assert np.max(np.abs((poly[:, None, None] * d).sum(0))) < tol
