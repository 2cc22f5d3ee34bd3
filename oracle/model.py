"""The coupled time step, as whole-array FP64 passes (oracle; test infrastructure only).

Order of one step (Sec. III B, summary after Eq. 55; the flow model is delegated to Refs. [13,29]):

  1. moments       rho = sum f, j = sum e f, T = sum g
  2. EOS           p_EOS, (dp/dT)_rho (Eq. 56); psi (READING: psi^2 = 2 (p_EOS - rho/3) / G)
  3. force         F = F_int + F_ads + F_b  (F_b = (rho - rho_ave) g, Sec. IV B; optionally, under an
                   open top, F_b = (rho - rho_top) g with rho_top the density held there)
  4. velocity      v = (j + F/2) / rho
  5. gradients     isotropic differences for grad T, lap T, grad rho, div v (after Eq. 55)
  6. source        phi (Eq. 28, underlined terms), S0 = phi + 0.5 d_t phi (Eq. 46), backward difference
  7. flow collide  MRT with forcing in moment space (READING of Refs. [13,29])
  8. heat collide  m* = m - Lambda (m - m_eq) + S (Eq. 45), m_eq of Eq. 53, corrections Eqs. 54-55
  9. stream        Eq. 47, periodic wrap
 10. boundaries    Zou-He wall / pressure rows (READING of Sec. IV A, Ref. [51]), Dirichlet T
 11. rho_ave       domain mean of this step's rho, used by the next step's buoyancy (READING)

State between steps: post-stream, post-boundary populations f and g at time t, phi(t - dt), and
rho_ave. Lattice units: dt = dx = 1, c_s^2 = 1/3.

READINGS (the paper is silent or delegates; every one is also listed in the design notes):
  * G = -1 and F_int = -G psi(x) sum_a w(|e_a|^2) psi(x + e_a) e_a with w(1) = 1/3, w(2) = 1/12.
  * The forcing scheme is the MRT forcing of Li, Luo & Li: v = (j + F/2)/rho,
    m* = m - Lambda (m - m_eq) + (I - Lambda/2) S_F with the sigma term in the energy moments.
  * Isotropic differences: d_i X = 3 sum_a w_a X(x+e_a) e_ai, lap X = 6 sum_a w_a (X(x+e_a) - X(x)).
  * First step: phi(t - dt) := phi(t). rho_ave lags one step (step 0 uses the initial mean).
  * x is periodic. A non-periodic y edge is an on-node row: a no-slip wall (Zou-He, v = 0 for the
    forcing scheme's velocity, so j = -F/2 with the wall row's force of the step before) or a
    fixed-density edge (Zou-He, u_x = 0). Stencils that cross such an edge, F_int's included, see
    ghost rows that copy the edge row (zero gradient), so a wall with G_w = 0 is neutral; at the y-
    wall the adsorption force F_ads = -G_w psi(x) sum_a w_a psi(x) s(x + e_a) e_a (s = 1 on the solid
    ghost row, which takes the fluid node's psi) sets the wettability (G_w < 0 attracts liquid). A y+ wall is a neutral lid: every solid
    surface of Sec. IV (the droplet on a surface, the heated wall) is the bottom one.
  * A held temperature on a non-periodic y edge (wall rows, the heated strip) enters through the
    unknown g by anti-bounce-back; without one those g bounce back (zero heat flux). A Dirichlet
    ring inside a periodic domain resets its nodes to g := M^{-1} m_eq(T_bc, v = 0).

Test hooks (never used by the GPU path): ``frozen_flow=(vx, vy)`` keeps f fixed and imposes a
uniform v with F = 0; ``frozen_thermal=True`` keeps g fixed; ``body_force=(ax, ay)`` adds the force
rho * (ax, ay), which drives a fluid of uniform density (plane Poiseuille flow).
"""

from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np

from . import eos
from . import lattice as L

EDGES = ("x-", "x+", "y-", "y+")


class OracleNonPhysical(RuntimeError):
    """Raised when rho <= 0, rho >= 1/b, T <= 0, psi^2 < 0 or a non-finite value appears."""

    def __init__(self, step, x, y, what):
        super().__init__(f"non-physical state at step {step}, node (x={x}, y={y}): {what}")
        self.step, self.x, self.y, self.what = step, x, y, what


@dataclass
class OracleParams:
    nx: int
    ny: int
    a: float = 3.0 / 49.0
    b: float = 2.0 / 21.0
    R: float = 1.0
    omega: float = 0.344
    G: float = -1.0
    s_f: Tuple[float, ...] = (1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25)
    s_g: Tuple[float, ...] = (1.0,) * 9
    sigma: float = 0.1
    lambda_mode: str = "const"  # "const": lambda fixed; "rho_cv_chi": lambda = rho c_V chi
    lam: float = 2.0 / 3.0
    chi: float = 0.06
    cV: float = 5.0
    gx: float = 0.0
    gy: float = 0.0
    buoyancy: int = 0  # 0 none; 1 (or True): reference rho_ave; 2: reference rho_bc of the y+ pressure edge
    flow_bc: Tuple[str, str, str, str] = ("periodic",) * 4  # x-, x+, y-, y+: periodic | wall | pressure
    rho_bc: Tuple[float, float, float, float] = (0.0,) * 4
    t_bc: Tuple[str, str, str, str] = ("none",) * 4  # none | dirichlet
    T_bc: Tuple[float, float, float, float] = (0.0,) * 4
    strip: Optional[Tuple[int, int, float]] = None  # heated strip on the y- row: [x0, x1) at T
    G_wall: float = 0.0
    model: str = "improved"  # improved | compromised | gong_cheng
    frozen_flow: Optional[Tuple[float, float]] = None
    body_force: Optional[Tuple[float, float]] = None
    frozen_thermal: bool = False

    def check(self):
        if self.flow_bc[0] != "periodic" or self.flow_bc[1] != "periodic":
            raise ValueError("x must be periodic")
        if (self.flow_bc[2] == "periodic") != (self.flow_bc[3] == "periodic"):
            raise ValueError("y edges must be both periodic or both non-periodic")
        if self.strip is not None and self.t_bc[2] != "dirichlet":
            raise ValueError("a heated strip needs a Dirichlet y- edge")
        if int(self.buoyancy) not in (0, 1, 2) or (int(self.buoyancy) == 2 and self.flow_bc[3] != "pressure"):
            raise ValueError("buoyancy is 0, 1, or 2 with a pressure y+ edge")
        if self.model not in ("improved", "compromised", "gong_cheng"):
            raise ValueError(self.model)


@dataclass
class OracleState:
    f: np.ndarray  # (9, ny, nx) post-stream density populations at time t
    g: np.ndarray  # (9, ny, nx) post-stream temperature populations at time t
    phi_prev: Optional[np.ndarray]  # phi(t - dt); None before the first step
    rho_ave: float
    step: int = 0
    last: dict = field(default_factory=dict)  # macroscopic fields of the last completed step


# ---------------------------------------------------------------------------------------------
# equilibria
# ---------------------------------------------------------------------------------------------


def flow_meq(rho, vx, vy):
    """Flow equilibrium moments rho(1, -2+3|v|^2, 1-3|v|^2, vx, -vx, vy, -vy, vx^2-vy^2, vx vy).

    READING: standard D2Q9 MRT equilibria of the delegated flow model (Refs. [13,29]).
    """
    v2 = vx * vx + vy * vy
    return np.stack([rho, rho * (-2.0 + 3.0 * v2), rho * (1.0 - 3.0 * v2), rho * vx, -rho * vx,
                     rho * vy, -rho * vy, rho * (vx * vx - vy * vy), rho * vx * vy])


def heat_meq(T, vx, vy, model):
    """Thermal equilibrium moments: Eq. 53, T(1,-2,2,vx,-vx,vy,-vy,0,0), for the improved model;
    Eq. 44, T(1,-2,1,vx,-vx,vy,-vy,0,0), for the compromised model (READING, Sec. IV); for the
    Gong-Cheng model the moments of Eq. 14, w T [1 + e.v/c_s^2 + vv:(ee - c_s^2 I)/(2 c_s^4)], which
    are those of the second-order equilibrium with rho replaced by T."""
    z = np.zeros_like(T)
    if model == "gong_cheng":
        return flow_meq(T, vx, vy)
    m2 = 2.0 * T if model == "improved" else T
    return np.stack([T, -2.0 * T, m2, T * vx, -T * vx, T * vy, -T * vy, z, z])


def init_state(p: OracleParams, rho, T, ux=None, uy=None) -> OracleState:
    """Initial populations f = M^{-1} m_eq(rho, u), g = M^{-1} m_eq(T, u) (equilibrium start),
    closed once by the boundary step so that the state, like every later one, holds post-boundary
    populations (READING: the paper does not state how the initial state meets the boundaries)."""
    p.check()
    rho = np.asarray(rho, dtype=np.float64).reshape(p.ny, p.nx)
    T = np.asarray(T, dtype=np.float64).reshape(p.ny, p.nx)
    ux = np.zeros_like(rho) if ux is None else np.asarray(ux, dtype=np.float64).reshape(p.ny, p.nx)
    uy = np.zeros_like(rho) if uy is None else np.asarray(uy, dtype=np.float64).reshape(p.ny, p.nx)
    f = flow_boundaries(p, L.from_moments(flow_meq(rho, ux, uy)))
    g = heat_boundaries(p, L.from_moments(heat_meq(T, ux, uy, p.model)))
    return OracleState(f=f, g=g, phi_prev=None, rho_ave=float(np.mean(f.sum(axis=0))))


# ---------------------------------------------------------------------------------------------
# neighbour access with the ghost rule for non-periodic y edges
# ---------------------------------------------------------------------------------------------


def _extend(X, p: OracleParams, ghost="copy"):
    """Pad a (ny, nx) field by one node: x wraps; y wraps when periodic, else ghost rows copy the
    edge row ('copy') or are zero ('zero')."""
    Xe = np.pad(X, ((0, 0), (1, 1)), mode="wrap")
    if p.flow_bc[2] == "periodic":
        return np.pad(Xe, ((1, 1), (0, 0)), mode="wrap")
    if ghost == "copy":
        return np.pad(Xe, ((1, 1), (0, 0)), mode="edge")
    return np.pad(Xe, ((1, 1), (0, 0)), mode="constant", constant_values=0.0)


def _nb(Xe, a):
    """X(x + e_a) from a one-node padded field."""
    ny, nx = Xe.shape[0] - 2, Xe.shape[1] - 2
    dx, dy = int(L.EX[a]), int(L.EY[a])
    return Xe[1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]


def grad(X, p):
    """Isotropic gradient (READING of the cited Eqs. (73)-(74)): d_i X = (1/c_s^2) sum_a w_a X(x+e_a) e_ai."""
    Xe = _extend(X, p)
    gx = sum(L.W[a] * _nb(Xe, a) * L.EX[a] for a in range(1, 9)) / L.CS2
    gy = sum(L.W[a] * _nb(Xe, a) * L.EY[a] for a in range(1, 9)) / L.CS2
    return gx, gy


def laplacian(X, p):
    """Isotropic Laplacian (READING): lap X = (2/c_s^2) sum_a w_a (X(x+e_a) - X(x))."""
    Xe = _extend(X, p)
    return 2.0 * sum(L.W[a] * (_nb(Xe, a) - X) for a in range(1, 9)) / L.CS2


# ---------------------------------------------------------------------------------------------
# the step
# ---------------------------------------------------------------------------------------------


def _check(p, s, rho, T, psi2):
    bad = ~np.isfinite(rho) | ~np.isfinite(T) | ~np.isfinite(psi2)
    bad |= (rho <= 0) | (rho * p.b >= 1.0) | (T <= 0) | (psi2 < 0)
    if np.any(bad):
        y, x = np.argwhere(bad)[0]
        raise OracleNonPhysical(s.step, int(x), int(y), f"rho={rho[y, x]!r} T={T[y, x]!r} psi2={psi2[y, x]!r}")


def macroscopic(p: OracleParams, s: OracleState):
    """Steps 1-6 of the step: moments, EOS, force, velocity, gradients and the source phi."""
    f, g = s.f, s.g
    # 1. moments (the flow model of Refs. [13,29]; T = sum g, Sec. II B)
    rho = f.sum(axis=0)
    jx = np.tensordot(L.EX.astype(float), f, axes=1)
    jy = np.tensordot(L.EY.astype(float), f, axes=1)
    T = g.sum(axis=0)
    # 2. EOS (Eq. 56) and the pseudopotential
    with np.errstate(all="ignore"):
        pe = eos.pressure(rho, T, p.a, p.b, p.R, p.omega)
        dpdT = eos.dp_dT(rho, T, p.a, p.b, p.R, p.omega)
        psi2 = eos.psi_squared(rho, pe, p.G)
    _check(p, s, rho, T, psi2)
    psi = np.sqrt(psi2)
    if p.frozen_flow is not None:
        vx = np.full_like(rho, p.frozen_flow[0])
        vy = np.full_like(rho, p.frozen_flow[1])
        Fx = Fy = Fix = Fiy = np.zeros_like(rho)
    else:
        # 3. force: pseudopotential interaction, adsorption at walls, buoyancy (Sec. IV B)
        pse = _extend(psi, p, ghost="copy")
        solid = np.zeros_like(pse)
        if p.flow_bc[2] == "wall":  # the wettable surface is the y- wall only (a y+ wall is neutral)
            solid[0, :] = 1.0
        wF = {1: 1.0 / 3.0, 2: 1.0 / 12.0}
        sx = sum(wF[L.EX[a] ** 2 + L.EY[a] ** 2] * _nb(pse, a) * L.EX[a] for a in range(1, 9))
        sy = sum(wF[L.EX[a] ** 2 + L.EY[a] ** 2] * _nb(pse, a) * L.EY[a] for a in range(1, 9))
        Fix, Fiy = -p.G * psi * sx, -p.G * psi * sy
        ax = sum(wF[L.EX[a] ** 2 + L.EY[a] ** 2] * _nb(solid, a) * L.EX[a] for a in range(1, 9))
        ay = sum(wF[L.EX[a] ** 2 + L.EY[a] ** 2] * _nb(solid, a) * L.EY[a] for a in range(1, 9))
        # F_ads = -G_w psi(x) sum_a w_a psi(x) s(x + e_a) e_a: the solid node takes the fluid node's psi
        Fx = Fix - p.G_wall * psi * psi * ax
        Fy = Fiy - p.G_wall * psi * psi * ay
        if p.buoyancy:
            # F_b = (rho - rho_ref) g: rho_ref = rho_ave (Sec. IV B), or for an open top the density it holds
            rho_ref = p.rho_bc[3] if p.buoyancy == 2 else s.rho_ave
            Fx = Fx + (rho - rho_ref) * p.gx
            Fy = Fy + (rho - rho_ref) * p.gy
        if p.body_force is not None:
            Fx = Fx + rho * p.body_force[0]
            Fy = Fy + rho * p.body_force[1]
        # 4. velocity including half the force
        vx = (jx + 0.5 * Fx) / rho
        vy = (jy + 0.5 * Fy) / rho
    # 5. isotropic differences (after Eq. 55)
    gTx, gTy = grad(T, p)
    lapT = laplacian(T, p)
    gvx, _ = grad(vx, p)
    _, gvy = grad(vy, p)
    divv = gvx + gvy
    # 6. source phi: the underlined terms of Eq. 28, with k = (1/s_3 - 1/2) c_s^2 (Eq. 41, A13)
    rcv = rho * p.cV
    if p.lambda_mode == "const":
        div_lam_gradT = p.lam * lapT
    else:  # lambda = rho c_V chi: div(lambda grad T) = lambda lap T + grad lambda . grad T (Sec. IV A)
        grx, gry = grad(rho, p)
        div_lam_gradT = rcv * p.chi * lapT + p.cV * p.chi * (grx * gTx + gry * gTy)
    if p.model == "gong_cheng":
        # Eq. 13: the Gong-Cheng source keeps only the compression term; conduction is left to the
        # LB diffusivity chi = (tau_g - 1/2) c_s^2 with tau_g = lambda/(rho c_s^2 c_V) + 1/2 (Sec. IV A)
        phi = T * (1.0 - dpdT / rcv) * divv
        lam = p.lam if p.lambda_mode == "const" else rcv * p.chi
        tau_g = lam / (rho * L.CS2 * p.cV) + 0.5
    else:
        k = (1.0 / p.s_g[3] - 0.5) * L.CS2
        phi = div_lam_gradT / rcv - k * lapT + T * (1.0 - dpdT / rcv) * divv
        tau_g = None
    return dict(rho=rho, jx=jx, jy=jy, T=T, p=pe, dpdT=dpdT, psi=psi, Fx=Fx, Fy=Fy, Fix=Fix, Fiy=Fiy,
                vx=vx, vy=vy, gTx=gTx, gTy=gTy, lapT=lapT, divv=divv, phi=phi, tau_g=tau_g)


def collide_flow(p: OracleParams, f, mac):
    """Flow MRT collision with forcing (READING of the improved pseudopotential model, Refs. [13,29]).

    m* = m - Lambda_f (m - m_eq) + (I - Lambda_f/2) S_F, with
    S_F = (0, 6 v.F + Q, -6 v.F - Q, Fx, -Fx, Fy, -Fy, 2(vx Fx - vy Fy), vx Fy + vy Fx),
    Q = 12 sigma |F_int|^2 / (psi^2 (1/s_e - 1/2)).
    """
    rho, vx, vy, Fx, Fy = mac["rho"], mac["vx"], mac["vy"], mac["Fx"], mac["Fy"]
    m = L.to_moments(f)
    meq = flow_meq(rho, vx, vy)
    s = np.asarray(p.s_f, dtype=np.float64)
    vF = vx * Fx + vy * Fy
    Q = 12.0 * p.sigma * (mac["Fix"] ** 2 + mac["Fiy"] ** 2) / (mac["psi"] ** 2 * (1.0 / s[1] - 0.5))
    z = np.zeros_like(rho)
    SF = np.stack([z, 6.0 * vF + Q, -6.0 * vF - Q, Fx, -Fx, Fy, -Fy, 2.0 * (vx * Fx - vy * Fy), vx * Fy + vy * Fx])
    mstar = m - s[:, None, None] * (m - meq) + (1.0 - 0.5 * s)[:, None, None] * SF
    return L.from_moments(mstar)


def collide_heat(p: OracleParams, g, mac, S0):
    """Thermal MRT collision, Eqs. 45-46 with m_eq of Eq. 53, then the corrections of Eqs. 54-55.

    m* = m - Lambda (m - m_eq) + (S0, 0, ..., 0);
    m3* += (1 - s3/2) s4 m4^(1),  m5* += (1 - s5/2) s6 m6^(1),  with dt m^(1) ~ m - m_eq (dt = 1).
    The compromised model (Sec. IV) omits both corrections; the Gong-Cheng model (Eqs. 12-14) is BGK.
    """
    T, vx, vy = mac["T"], mac["vx"], mac["vy"]
    m = L.to_moments(g)
    meq = heat_meq(T, vx, vy, p.model)
    if p.model == "gong_cheng":
        # Eq. 12: BGK with the local tau_g, source G_a = w_a phi (moments phi (1, -2, 1, 0, ..., 0))
        G = np.zeros_like(m)
        G[0], G[1], G[2] = S0, -2.0 * S0, S0
        return L.from_moments(m - (m - meq) / mac["tau_g"] + G)
    s = np.asarray(p.s_g, dtype=np.float64)
    mstar = m - s[:, None, None] * (m - meq)
    mstar[0] = mstar[0] + S0
    if p.model == "improved":
        mstar[3] = mstar[3] + (1.0 - 0.5 * s[3]) * s[4] * (m[4] - meq[4])
        mstar[5] = mstar[5] + (1.0 - 0.5 * s[5]) * s[6] * (m[6] - meq[6])
    return L.from_moments(mstar)


def stream(pop):
    """Eq. 47: pop_a(x + e_a, t + dt) = pop*_a(x, t), with periodic wrap on both axes (the rows a
    non-periodic edge receives through the wrap are unknowns that the boundary step overwrites)."""
    out = np.empty_like(pop)
    for a in range(9):
        out[a] = np.roll(np.roll(pop[a], int(L.EY[a]), axis=0), int(L.EX[a]), axis=1)
    return out


def flow_boundaries(p: OracleParams, f, F=None):
    """Zou-He closures on non-periodic y edges (READING of Ref. [51]; u = 0 at a wall, u_x = 0 and
    rho = rho_bc at a pressure edge). Unknowns at y- are f2, f5, f6; at y+ they are f4, f7, f8.

    At a wall the closure sets the momentum j = sum e f to -F/2, so that the velocity of the forcing
    scheme, v = (j + F/2)/rho, vanishes there (READING: with j = 0 a force on the wall row, such as
    the adsorption force, moves the fluid through the wall at F/(2 rho) and the wall drains mass).
    F = (Fx, Fy) is the force of the step that produced f, one step behind the step that will use
    the closed state; None (the initial state) means F = 0."""
    for edge, row in (("y-", 0), ("y+", -1)):
        kind = p.flow_bc[EDGES.index(edge)]
        if kind == "periodic":
            continue
        q = [f[a, row].copy() for a in range(9)]
        d13 = q[1] - q[3]
        if kind == "wall":
            jx = np.zeros_like(q[0]) if F is None else -0.5 * F[0][row]
            jy = np.zeros_like(q[0]) if F is None else -0.5 * F[1][row]
        if edge == "y-":
            if kind == "wall":  # Zou-He for a prescribed j: f2 - f4 = 2/3 j_y, and j_x from f5 - f6
                f[2, row] = q[4] + 2.0 / 3.0 * jy
                f[5, row] = q[7] - 0.5 * d13 + 0.5 * jx + jy / 6.0
                f[6, row] = q[8] + 0.5 * d13 - 0.5 * jx + jy / 6.0
            else:
                rb = p.rho_bc[2]
                ru = rb - (q[0] + q[1] + q[3] + 2.0 * (q[4] + q[7] + q[8]))  # rho_bc * u_y
                f[2, row] = q[4] + 2.0 / 3.0 * ru
                f[5, row] = q[7] - 0.5 * d13 + ru / 6.0
                f[6, row] = q[8] + 0.5 * d13 + ru / 6.0
        else:
            if kind == "wall":
                f[4, row] = q[2] - 2.0 / 3.0 * jy
                f[7, row] = q[5] + 0.5 * d13 - 0.5 * jx - jy / 6.0
                f[8, row] = q[6] - 0.5 * d13 + 0.5 * jx - jy / 6.0
            else:
                rb = p.rho_bc[3]
                ru = (q[0] + q[1] + q[3] + 2.0 * (q[2] + q[5] + q[6])) - rb  # rho_bc * u_y
                f[4, row] = q[2] - 2.0 / 3.0 * ru
                f[7, row] = q[5] + 0.5 * d13 - ru / 6.0
                f[8, row] = q[6] - 0.5 * d13 - ru / 6.0
    return f


def _heat_eq_at_rest(T, model):
    z = np.zeros_like(T)
    return L.from_moments(heat_meq(T, z, z, model))


def _row_T(p: OracleParams, edge, n):
    T = np.full(n, p.T_bc[edge])
    if edge == 2 and p.strip is not None:
        x0, x1, Ts = p.strip
        T[x0:x1] = Ts
    return T


def heat_boundaries(p: OracleParams, g):
    """Thermal boundary step (READING; the paper states only which temperatures are held).

    On a non-periodic y edge the unknown g (those streamed in from beyond the edge) are closed by
    bounce-back: g_a = -g_opp(a) + 2 g_a^eq(T_bc, 0) when the edge holds T_bc (anti-bounce-back, so
    heat enters through the wall), g_a = g_opp(a) otherwise (zero heat flux). Dirichlet edges of a
    periodic axis (a ring of nodes inside a periodic domain) reset the node to g := M^{-1} m_eq(T_bc, 0):
    x edges first, then y edges."""
    ny, nx = g.shape[1:]
    if p.flow_bc[2] != "periodic":
        for edge, row, unknown, known in ((2, 0, (2, 5, 6), (4, 7, 8)), (3, -1, (4, 7, 8), (2, 5, 6))):
            if p.t_bc[edge] == "dirichlet":
                geq = _heat_eq_at_rest(_row_T(p, edge, nx), p.model)
                for a, b in zip(unknown, known):
                    g[a, row] = -g[b, row] + 2.0 * geq[a]
            else:
                for a, b in zip(unknown, known):
                    g[a, row] = g[b, row]
    if p.t_bc[0] == "dirichlet":
        g[:, :, 0] = _heat_eq_at_rest(np.full(ny, p.T_bc[0]), p.model)
    if p.t_bc[1] == "dirichlet":
        g[:, :, -1] = _heat_eq_at_rest(np.full(ny, p.T_bc[1]), p.model)
    if p.flow_bc[2] == "periodic":
        if p.t_bc[2] == "dirichlet":
            g[:, 0, :] = _heat_eq_at_rest(_row_T(p, 2, nx), p.model)
        if p.t_bc[3] == "dirichlet":
            g[:, -1, :] = _heat_eq_at_rest(_row_T(p, 3, nx), p.model)
    return g


def step(p: OracleParams, s: OracleState) -> OracleState:
    """Advance the state by one time step (steps 1-11 of the module docstring)."""
    mac = macroscopic(p, s)
    phi = mac["phi"]
    phi_prev = phi if s.phi_prev is None else s.phi_prev
    if p.model == "improved":
        S0 = phi + 0.5 * (phi - phi_prev)  # Eq. 46 with d_t phi ~ [phi(t) - phi(t - dt)] / dt
    else:
        S0 = phi
    if p.frozen_flow is not None:
        fn = s.f
    else:
        fn = flow_boundaries(p, stream(collide_flow(p, s.f, mac)), (mac["Fx"], mac["Fy"]))
    gn = s.g if p.frozen_thermal else heat_boundaries(p, stream(collide_heat(p, s.g, mac, S0)))
    return OracleState(f=fn, g=gn, phi_prev=phi, rho_ave=float(np.mean(mac["rho"])), step=s.step + 1, last=mac)


def run(p: OracleParams, s: OracleState, n: int) -> OracleState:
    for _ in range(n):
        s = step(p, s)
    return s


def fields(p: OracleParams, s: OracleState):
    """rho, u_x, u_y, T of the current state; u = (sum e f + F/2)/rho as the step would compute it."""
    mac = macroscopic(p, s)
    return mac["rho"], mac["vx"], mac["vy"], mac["T"]
