"""Pins of the oracle's no-slip wall (Zou-He closure for a prescribed momentum, j = -F/2, so that the
forcing scheme's velocity v = (j + F/2)/rho vanishes on the wall row).

- Plane Poiseuille flow: a uniform fluid between the two on-node walls y = 0 and y = H = ny - 1, driven
  by a uniform body force rho * a_x, reaches u_x(y) = a_x y (H - y) / (2 nu). This is the textbook
  closed form. A closure with j = 0 instead leaves the wall slipping at a_x / 2 (5e-3 of the peak here).
  A wrong sign or factor in the tangential target fails it too.
- A liquid at rest on a wettable wall (adsorption force normal to the wall row), in a closed box with
  gravity, keeps its mass. A closure with j = 0 moves the liquid through the wall at F/(2 rho) and
  drains the box: about 0.4 mass units per step here, the whole mass in 1600 steps.
- A sessile droplet meets a wall without adsorption at 90 degrees, and the adsorption force moves the
  angle the right way: above 90 for G_w > 0, below for G_w < 0."""

import numpy as np
import pytest

from oracle import model
from paper_1709_04400_gb300 import inputs

from .helpers import RL, RV, TS, contact_angle


def test_plane_poiseuille_between_walls():
    nx, ny, a = 4, 10, 1e-6
    p = model.OracleParams(nx=nx, ny=ny, flow_bc=("periodic", "periodic", "wall", "wall"), body_force=(a, 0.0))
    s = model.init_state(p, np.full((ny, nx), RL), np.full((ny, nx), TS))
    s = model.run(p, s, 2500)
    rho, ux, uy, _ = model.fields(p, s)
    y = np.arange(ny, dtype=float)
    nu = (1.0 / p.s_f[7] - 0.5) / 3.0
    exact = a * y * (ny - 1 - y) / (2.0 * nu)
    assert np.max(np.abs(ux - exact[:, None])) <= 1e-8 * exact.max()
    assert np.max(np.abs(uy)) <= 1e-9 * exact.max()
    assert np.max(np.abs(ux[0])) <= 1e-8 * exact.max() and np.max(np.abs(ux[-1])) <= 1e-8 * exact.max()


def test_wettable_wall_keeps_the_liquid():
    nx, ny = 8, 24
    p = model.OracleParams(nx=nx, ny=ny, flow_bc=("periodic", "periodic", "wall", "wall"), G_wall=-0.2,
                           buoyancy=True, gy=-3e-5, t_bc=("none", "none", "dirichlet", "dirichlet"),
                           T_bc=(0.0, 0.0, TS, TS), lambda_mode="rho_cv_chi", chi=0.06)
    rho, T = inputs.pool_with_noise(3, nx, ny, 4, RL, RV, TS, amp=0.0)
    s = model.init_state(p, rho, T)
    m0 = s.f.sum()
    s = model.run(p, s, 2000)
    m2000 = s.f.sum()
    s = model.run(p, s, 1000)
    m3000 = s.f.sum()
    _, _, uy, _ = model.fields(p, s)
    # the wall row's density settles once (the closure's rho includes -F_y/2), then holds
    assert abs(m3000 - m0) <= 5e-3 * m0
    assert abs(m3000 - m2000) <= 1e-4 * m0
    # F_y / (2 rho) on the wall row is about 1.6e-2; the wall row is at rest to the transient's decay
    assert np.max(np.abs(uy[0])) <= 1e-6


@pytest.mark.parametrize("G_wall,lo,hi", [(0.0, 87.0, 93.0), (0.1, 105.0, 125.0), (-0.1, 55.0, 75.0)],
                         ids=["neutral", "repelling", "wetting"])
def test_sessile_droplet_contact_angle(G_wall, lo, hi):
    """A droplet (r = 15) on the y- wall of an 80 x 50 box, isothermal, after 2000 steps. A wall
    without adsorption, whose ghost row copies the edge row, meets the interface at 90 degrees. G_w > 0
    repels the liquid (angle above 90: 113.7 here) and G_w < 0 attracts it (66.6 here). A sign error or
    a dropped factor in F_ads fails one of the three."""
    nx, ny = 80, 50
    rho = inputs.tanh_droplet(nx, ny, 15.0, 4.0, RL, RV, cx=nx / 2.0, cy=4.0)
    p = model.OracleParams(nx=nx, ny=ny, flow_bc=("periodic", "periodic", "wall", "pressure"), rho_bc=(0, 0, 0, RV),
                           t_bc=("none", "none", "dirichlet", "dirichlet"), T_bc=(0, 0, TS, TS), G_wall=G_wall,
                           lambda_mode="rho_cv_chi", chi=0.08)
    s = model.run(p, model.init_state(p, rho, np.full((ny, nx), TS)), 2000)
    theta = contact_angle(model.fields(p, s)[0])
    assert lo <= theta <= hi, theta


@pytest.mark.parametrize("mode", [1, 2], ids=["rho_ave", "rho_top"])
def test_pool_under_an_open_top(mode):
    """A liquid pool at rest under a vapour layer with an open, fixed-density top and gravity. With the
    reference density held at the top (mode 2) the pool reaches hydrostatic rest: the vapour at the top
    is force-free and the liquid's weight is carried by the wall. With the domain mean as the reference
    (mode 1, meant for closed domains) the vapour is pushed upward with nothing to hold it, and a steady
    outflow through the top drains the pool."""
    nx, ny = 8, 60
    p = model.OracleParams(nx=nx, ny=ny, flow_bc=("periodic", "periodic", "wall", "pressure"), rho_bc=(0, 0, 0, RV),
                           t_bc=("none", "none", "dirichlet", "dirichlet"), T_bc=(0, 0, TS, TS), buoyancy=mode,
                           gy=-3e-5, lambda_mode="rho_cv_chi", chi=0.06)
    rho, T = inputs.pool_with_noise(3, nx, ny, 4, RL, RV, TS, amp=0.0)
    s = model.run(p, model.init_state(p, rho, T), 3000)
    m3000 = s.f.sum()
    s = model.run(p, s, 3000)
    rho_f, ux, uy, _ = model.fields(p, s)
    drift = (s.f.sum() - m3000) / m3000
    if mode == 2:
        assert np.max(np.abs(uy)) < 1e-4 and abs(drift) < 1e-4, (np.max(np.abs(uy)), drift)
        # the pressure edge holds what it prescribes: rho = rho_bc and u_x = 0 on the top row
        assert np.max(np.abs(rho_f[-1] / RV - 1.0)) < 1e-13 and np.max(np.abs(ux[-1])) < 1e-15
    else:
        assert np.mean(uy[-1]) > 2e-4 and drift < -1e-3, (np.mean(uy[-1]), drift)


def test_steady_conduction_between_held_rows():
    """Held temperatures (anti-bounce-back of the unknown g on the wall rows): between rows held at
    T_lo and T_hi, a fluid at rest (the frozen-flow hook) reaches the linear conduction profile. Its
    interior, three nodes or more from either wall, is linear to 1e-4 of dT, as the steady diffusion
    equation requires. The heat flux is within 2 % of (T_hi - T_lo)/(ny - 1), and the wall rows sit within
    0.5 % of dT of their held values. A sign error in the closure (no heat enters) or a wrong equilibrium
    (a shifted wall temperature) fails it."""
    nx, ny = 4, 21
    T_lo, T_hi = 1.02 * TS, 0.98 * TS
    dT = T_lo - T_hi
    p = model.OracleParams(nx=nx, ny=ny, flow_bc=("periodic", "periodic", "wall", "wall"), frozen_flow=(0.0, 0.0),
                           t_bc=("none", "none", "dirichlet", "dirichlet"), T_bc=(0, 0, T_lo, T_hi),
                           lambda_mode="rho_cv_chi", chi=0.2)
    s = model.run(p, model.init_state(p, np.full((ny, nx), RL), np.full((ny, nx), TS)), 3000)
    T = model.fields(p, s)[3][:, 0]
    y = np.arange(ny)
    c = np.polyfit(y[3:-3], T[3:-3], 1)
    assert np.max(np.abs(np.polyval(c, y[3:-3]) - T[3:-3])) < 1e-4 * dT
    assert abs(c[0] / ((T_hi - T_lo) / (ny - 1)) - 1.0) < 0.02
    assert abs(T[0] - T_lo) < 5e-3 * dT and abs(T[-1] - T_hi) < 5e-3 * dT
