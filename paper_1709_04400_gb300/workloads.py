"""The synthetic workloads, as plain parameter sets plus seeded initial fields.

A case is a dict whose keys name the physical set-up (grid, boundary kinds as strings, rates,
conductivity, gravity, boundary values) and two FP64 arrays rho, T. Temperatures and densities
that depend on the equation of state (T_c, coexistence densities) are arguments, so the caller
decides whose EOS evaluation supplies them. Nothing here evaluates the lattice Boltzmann method.

  droplet_periodic     128 x 128 periodic, droplet R = 25 (tanh width 4) between the coexistence
                       densities at 0.86 T_c, T = 0.86 T_c + seeded 0.01 T_c sinusoid, u = 0,
                       lambda = 2/3, c_V = 5, nu = 0.1 (Sec. IV A parameters).
  droplet_evaporation  256 x 256, droplet R = 40 at T_s = 0.86 T_c, outer ring held at T_s + dT
                       (dT / T_c in {0.05, 0.1, 0.2}); periodic flow; lambda = 2/3 (Sec. IV A).
  heated_wall          300 x 400 pool (liquid below y = 200, vapour above, density noise +-1e-4),
                       no-slip bottom wall at T_s with a heated strip 20 nodes wide at T_s + 0.3 T_c,
                       top held at the vapour density and T_s, g = 3e-5 downward with buoyancy relative
                       to the top's density, lambda = rho c_V chi with chi = 0.06 (Sec. IV B).
  paper_d2_law         the paper's own D^2-law set-up (Sec. IV A): 200 x 200, D0 = 60, dT = 0.14 T_c.
  bubble_departure     100 x 200 closed pool under a thin vapour cushion, wettable wall with a heated
                       strip, g = 1e-4: bubbles grow, detach and repeat (Sec. IV B).
"""

import numpy as np

from . import inputs

NU = 0.1
S_NU = 1.0 / (3.0 * NU + 0.5)  # nu = c_s^2 (1/s_nu - 1/2)
BASE = dict(
    s_f=(1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, S_NU, S_NU),
    s_g=(1.0,) * 9,
    sigma=0.1,
    cV=5.0,
    model="improved",
)
# G_wall of the heated-wall case: a neutral wall (no fluid-solid force beyond the edge-copy ghosts); the
# paper's 45-degree contact angle is not calibrated. A wettable bottom wall (G_wall < 0) is stable too now
# that the wall closure holds v = 0 under the adsorption force.
HEATED_WALL_G_WALL = 0.0


def droplet_periodic(Tc, rho_v, rho_l, n=128, radius=25.0, seed=inputs.SEED_BASE):
    rho, T, info = inputs.droplet_periodic(seed, n, n, radius, 4.0, rho_l, rho_v, Tc)
    case = dict(BASE, name=f"droplet_periodic_{n}", nx=n, ny=n, lambda_mode="const", lam=2.0 / 3.0,
                flow_bc=("periodic",) * 4, t_bc=("none",) * 4)
    return case, rho, T


def droplet_evaporation(Tc, rho_v, rho_l, n=256, radius=40.0, dT_ratio=0.1):
    Ts = 0.86 * Tc
    dT = dT_ratio * Tc
    rho, T = inputs.droplet_hot_ring(n, n, radius, 4.0, rho_l, rho_v, Ts, dT)
    case = dict(BASE, name=f"droplet_evaporation_{n}_dT{dT_ratio:g}Tc", nx=n, ny=n, lambda_mode="const",
                lam=2.0 / 3.0, flow_bc=("periodic",) * 4, t_bc=("dirichlet",) * 4, T_bc=(Ts + dT,) * 4)
    return case, rho, T


def heated_wall(Tc, rho_v, rho_l, nx=300, ny=400, strip_width=20, dT_strip_ratio=0.3, g=3e-5,
                seed=inputs.SEED_BASE + 2, top="pressure", vapour_rows=None, buoyancy=None, G_wall=None):
    """top = "pressure" holds the vapour density (the fixed-pressure top); "wall" closes the pool.
    vapour_rows = None fills the pool to ny/2; a number leaves that many vapour rows under the top.
    buoyancy = 1 takes F_b = (rho - rho_ave) g (Sec. IV B); 2, with the pressure top, takes the density
    held there as the reference, under which an open top stays at rest. None: 2 under the pressure top
    (with 1 its vapour is pushed out and the run fails after about 1850 steps), 1 in a closed pool."""
    if buoyancy is None:
        buoyancy = 2 if top == "pressure" else 1
    Ts = 0.86 * Tc
    surface = None if vapour_rows is None else ny - vapour_rows
    rho, T = inputs.pool_with_noise(seed, nx, ny, 4.0, rho_l, rho_v, Ts, amp=1e-4, surface=surface)
    x0 = nx // 2 - strip_width // 2
    case = dict(BASE, name=f"heated_wall_{nx}x{ny}" + ("" if top == "pressure" else "_closed"), nx=nx, ny=ny,
                lambda_mode="rho_cv_chi", lam=0.0, chi=0.06, gx=0.0, gy=-g, buoyancy=buoyancy,
                flow_bc=("periodic", "periodic", "wall", top), rho_bc=(0.0, 0.0, 0.0, rho_v),
                t_bc=("none", "none", "dirichlet", "dirichlet"), T_bc=(0.0, 0.0, Ts, Ts),
                strip=(x0, x0 + strip_width, Ts + dT_strip_ratio * Tc),
                G_wall=HEATED_WALL_G_WALL if G_wall is None else G_wall)
    return case, rho, T


def bubble_departure(Tc, rho_v, rho_l, nx=100, ny=200, strip_width=20, dT_strip_ratio=0.3, g=1e-4,
                     G_wall=-0.1, surface_ratio=0.85, seed=inputs.SEED_BASE + 6):
    """Nucleate boiling with departing bubbles (Sec. IV B, closed pool): liquid below y = 0.85 ny under
    a thin vapour cushion, a wettable bottom wall at T_s (G_wall = -0.1) with a heated strip of 20 nodes
    at T_s + 0.3 T_c, a closed neutral lid at T_s, g = 1e-4 with buoyancy (rho - rho_ave) g, and
    lambda = rho c_V chi with chi = 0.06. The vapour over the strip grows into a bubble, which departs
    after about 9500 steps and leaves a small attached bubble that repeats the cycle."""
    Ts = 0.86 * Tc
    rho, T = inputs.pool_with_noise(seed, nx, ny, 4.0, rho_l, rho_v, Ts, amp=1e-4, surface=surface_ratio * ny)
    x0 = nx // 2 - strip_width // 2
    case = dict(BASE, name=f"bubble_departure_{nx}x{ny}", nx=nx, ny=ny, lambda_mode="rho_cv_chi", lam=0.0,
                chi=0.06, gx=0.0, gy=-g, buoyancy=True, flow_bc=("periodic", "periodic", "wall", "wall"),
                rho_bc=(0.0,) * 4, t_bc=("none", "none", "dirichlet", "dirichlet"), T_bc=(0.0, 0.0, Ts, Ts),
                strip=(x0, x0 + strip_width, Ts + dT_strip_ratio * Tc), G_wall=G_wall,
                surface=int(surface_ratio * ny))
    return case, rho, T


def droplet_on_surface(Tc, rho_v, rho_l, nx=300, ny=150, radius=40.0, G_wall=0.1, wall_T_ratio=None,
                       lambda_mode="rho_cv_chi", chi=0.08, lam=1.0, model="improved"):
    """A droplet on a solid surface (Sec. IV A, second test): a 300 x 150 domain, periodic in x, a
    droplet of radius 40 on the bottom wall (the circle's centre 12 nodes above it, near the cap of a
    108-degree contact angle), a non-wetting wall (G_wall > 0), an open top held at the vapour
    density and at T_s (the far vapour at saturation), no gravity, c_V = 5, nu = 0.1, lambda = rho c_V chi with chi = 0.08
    (or a constant lambda). wall_T_ratio = None holds the wall at T_s (the isothermal relaxation the
    paper runs first); 0.875 heats it to 0.875 T_c, which drives the evaporation."""
    Ts = 0.86 * Tc
    rho = inputs.tanh_droplet(nx, ny, radius, 4.0, rho_l, rho_v, cx=nx / 2.0, cy=12.0)
    T = np.full((ny, nx), Ts)
    Tw = Ts if wall_T_ratio is None else wall_T_ratio * Tc
    case = dict(BASE, name=f"droplet_on_surface_{nx}x{ny}", nx=nx, ny=ny, lambda_mode=lambda_mode,
                lam=lam if lambda_mode == "const" else 0.0, chi=chi, model=model,
                flow_bc=("periodic", "periodic", "wall", "pressure"), rho_bc=(0.0, 0.0, 0.0, rho_v),
                t_bc=("none", "none", "dirichlet", "dirichlet"), T_bc=(0.0, 0.0, Tw, Ts), G_wall=G_wall)
    return case, rho, T


def mixed_small(Tc, rho_v, rho_l, nx=37, ny=29, seed=inputs.SEED_BASE + 5):
    """Small ragged grid with every boundary class: wall bottom with a strip, pressure top,
    buoyancy, lambda = rho c_V chi, non-default thermal rates (every term of Eqs. 45-55 active)."""
    Ts = 0.86 * Tc
    rho, T = inputs.pool_with_noise(seed, nx, ny, 4.0, rho_l, rho_v, Ts, amp=0.01)
    case = dict(BASE, name=f"mixed_{nx}x{ny}", nx=nx, ny=ny, lambda_mode="rho_cv_chi", lam=0.0, chi=0.06,
                s_g=(1.0, 0.9, 1.05, 1.0, 1.2, 1.0, 1.2, 0.95, 0.85),
                gx=1e-5, gy=-3e-5, buoyancy=True,
                flow_bc=("periodic", "periodic", "wall", "pressure"), rho_bc=(0.0, 0.0, 0.0, rho_v),
                t_bc=("none", "none", "dirichlet", "dirichlet"), T_bc=(0.0, 0.0, Ts, Ts),
                strip=(nx // 4, nx // 2 + 1, Ts + 0.1 * Tc), G_wall=-0.2)
    return case, rho, T


def batched_evaporation(Tc, rho_v, rho_l, count=256, side_lo=64, side_hi=512, seed=inputs.SEED_BASE + 3):
    """Droplet-evaporation instances of uneven size: side uniform in {side_lo..side_hi}, radius
    uniform in [0.15, 0.3] of the side, superheat uniform in [0.05, 0.3] T_c (seeded)."""
    u = inputs.uniform(seed, 3 * count).reshape(count, 3)
    out = []
    for k in range(count):
        n = side_lo + int(u[k, 0] * (side_hi - side_lo + 1))
        radius = (0.15 + 0.15 * u[k, 1]) * n
        dT = 0.05 + 0.25 * u[k, 2]
        case, rho, T = droplet_evaporation(Tc, rho_v, rho_l, n=n, radius=radius, dT_ratio=dT)
        out.append((case, rho, T))
    return out



def paper_d2_law(Tc, rho_v, rho_l, model="improved", lam=2.0 / 3.0):
    """The droplet-evaporation set-up of Sec. IV A: 200 x 200, a droplet of diameter D0 = 60 at the centre,
    constant lambda (2/3 in the paper), superheat dT = 0.14 T_c in the vapour and on the boundaries,
    s3 = s5 = 1, c_V = 5, nu = 0.1, no gravity (flow periodic)."""
    case, rho, T = droplet_evaporation(Tc, rho_v, rho_l, n=200, radius=30.0, dT_ratio=0.14)
    return dict(case, name=f"paper_d2_law_{model}_lam{lam:.4g}", model=model, lam=lam), rho, T


def droplet_area(rho):
    """Droplet area from a density field: sum of clip((rho - rho_far)/(rho_centre - rho_far), 0, 1), with
    rho_far the mean of four near-corner nodes and rho_centre the centre node (self-normalising to the
    current phase densities)."""
    ny, nx = rho.shape
    lo = np.mean([rho[2, 2], rho[2, -3], rho[-3, 2], rho[-3, -3]])
    hi = rho[ny // 2, nx // 2]
    return float(np.clip((rho - lo) / (hi - lo), 0.0, 1.0).sum())


def vapour_volume(rho, rho_v, rho_l, rows):
    """Vapour volume in the lowest `rows` rows of a pool: sum of clip((rho_l - rho)/(rho_l - rho_v), 0, 1).
    Below the free surface of the heated-wall pool this is the vapour formed over the heater; it is a
    smooth function of the density, so it compares across precisions without a threshold's jumps."""
    r = np.asarray(rho)[:rows]
    return float(np.clip((rho_l - r) / (rho_l - rho_v), 0.0, 1.0).sum())
