"""Plain FP64 CPU oracle of the coupled pseudopotential-flow + improved thermal MRT-LB step.

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously correct statement of what the
GPU library computes, written from Li, Zhou & Yan, "Improved thermal lattice Boltzmann model
for simulation of liquid-vapor phase change" (arXiv:1709.04400). Only the tests, the smoke
check in ``__graft_entry__`` and the CPU-baseline / reference arm of ``bench.py`` may import
it. The GPU library never imports, links or calls anything here, and nothing here imports the
GPU library: the two share no code. Inputs come from ``paper_1709_04400_gb300.inputs``, a
module that holds random-number and initial-shape generation only.

Modules
-------
lattice  D2Q9 velocities, weights and the MRT transformation matrix (Eqs. 42-44).
eos      Peng-Robinson equation of state (Eq. 56), (dp/dT)_rho, psi, Maxwell coexistence.
model    The time step, whole-array passes in the order the paper states the model
         (Sec. III B summary after Eq. 55; Eqs. 45-47, 53-55; Eq. 28 source).

Every function cites the passage it follows. Where the paper delegates a detail to a reference
that is not reproduced in the paper (flow model, isotropic stencils, Zou-He, contact angle),
the reading taken is stated in the docstring and marked READING.

Pins (tests/test_oracle_*.py) check the oracle against what the paper and the mathematics fix. The
flow collision with forcing reduces, with every MRT rate equal and sigma = 0, to BGK with Guo's
forcing term, a textbook closed form checked node by node with v and F in both directions (every row
of S_F, the velocity-dependent ones included); the sigma term is checked to change only the two energy
moments, by the amounts its formula fixes, for an interaction force built in closed form. The
source phi is pinned term by term: conduction by the chi q^2 decay of a temperature mode and by the
constant heat content of a fluid at rest under a variable conductivity; the pressure work, and the
second-order time discretisation of Eq. 46, by the adiabatic temperature-density ratio of an acoustic
wave. Eqs. 54-55 are pinned by the spreading of heat advected by a uniform flow. The no-slip wall is pinned by plane Poiseuille flow, by the mass of a liquid on a wettable wall, by the
90-degree contact angle of a neutral wall, and by an open-top pool at hydrostatic rest. Held
temperatures (``heat_boundaries``) are pinned by steady conduction between held rows. The
fixed-density (pressure) edge is pinned by the values it prescribes (rho = rho_bc, u_x = 0 on its row)
and by the hydrostatic rest of a pool under it.
"""

from . import lattice, eos, model  # noqa: F401
from .model import OracleParams, OracleState, OracleNonPhysical, init_state, step, run, fields  # noqa: F401
