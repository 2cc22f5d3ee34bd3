"""Invariants of the oracle's coupled step that hold exactly (or to round-off) whatever the readings:
mass conservation and momentum balance on periodic domains (collision conserves m0 and adds F to
j; streaming permutes), translation invariance, mirror and x<->y symmetry of the D2Q9 scheme."""

import numpy as np
import pytest

from oracle import eos, model
from paper_1709_04400_gb300 import inputs

A, B, R, OM = 3.0 / 49.0, 2.0 / 21.0, 1.0, 0.344
TC = eos.critical_temperature(A, B, R)
TS = 0.86 * TC
RV, RL, _ = eos.maxwell_coexistence(TS, A, B, R, OM)


def _fields(nx, ny, seed=7):
    return inputs.random_fields(seed, nx, ny, RL, RV, TS, 0.05 * TC)


def _params(nx, ny, **kw):
    base = dict(nx=nx, ny=ny, s_g=(1.0, 0.9, 1.05, 1.0, 1.2, 1.0, 1.2, 0.95, 0.85))
    base.update(kw)
    return model.OracleParams(**base)


def test_mass_conservation_periodic_1000_steps():
    """Exact mass conservation on a periodic domain."""
    p = _params(32, 32, lambda_mode="rho_cv_chi", chi=0.06)
    rho, T, _ = inputs.droplet_periodic(inputs.SEED_BASE, 32, 32, 8, 4, RL, RV, TC)
    s = model.init_state(p, rho, T)
    m0 = s.f.sum()
    s = model.run(p, s, 1000)
    assert abs(s.f.sum() - m0) / m0 < 1e-13


def test_momentum_balance_periodic():
    """sum_x j(t+1) = sum_x j(t) + sum_x F and the pair force sums to zero: total momentum stays 0."""
    p = _params(24, 20, buoyancy=True, gy=-3e-5)
    rho, T = _fields(24, 20)
    s = model.init_state(p, rho, T)
    ex = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1.0])
    ey = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1.0])
    for _ in range(40):
        s = model.step(p, s)
        jx, jy = np.tensordot(ex, s.f, 1), np.tensordot(ey, s.f, 1)
        scale = np.abs(jx).sum() + np.abs(jy).sum()
        assert scale > 1e-3
        assert abs(jx.sum()) < 1e-12 * scale and abs(jy.sum()) < 1e-12 * scale


def test_translation_invariance():
    p = _params(24, 20)
    rho, T = _fields(24, 20)
    a = model.run(p, model.init_state(p, rho, T), 30)
    sh = (5, -3)
    b = model.run(p, model.init_state(p, np.roll(rho, sh, (0, 1)), np.roll(T, sh, (0, 1))), 30)
    assert np.array_equal(np.roll(a.f, sh, (1, 2)), b.f)
    assert np.array_equal(np.roll(a.g, sh, (1, 2)), b.g)


@pytest.mark.parametrize("walls", [False, True])
def test_x_mirror_symmetry(walls):
    """Mirroring x maps the solution onto its mirror image (e_a -> (-ex, ey)); with walls, a pressure
    top and a centred heated strip the set-up is mirror symmetric too."""
    nx, ny = 24, 20
    kw = {}
    if walls:
        kw = dict(flow_bc=("periodic", "periodic", "wall", "pressure"), rho_bc=(0, 0, 0, RV),
                  t_bc=("none", "none", "dirichlet", "dirichlet"), T_bc=(0, 0, TS, TS),
                  strip=(8, 16, TS + 0.2 * TC), G_wall=-0.3, buoyancy=True, gy=-3e-5,
                  lambda_mode="rho_cv_chi", chi=0.06)
    p = _params(nx, ny, **kw)
    if walls:  # liquid pool under vapour, consistent with the wall and the vapour-density top
        rho, T = inputs.pool_with_noise(3, nx, ny, 4, RL, RV, TS, amp=0.05)
    else:
        rho, T = _fields(nx, ny)
    a = model.run(p, model.init_state(p, rho, T), 30)
    b = model.run(p, model.init_state(p, rho[:, ::-1], T[:, ::-1]), 30)
    mir = [0, 3, 2, 1, 4, 6, 5, 8, 7]
    assert np.allclose(a.f[mir][:, :, ::-1], b.f, rtol=1e-11, atol=1e-13)
    assert np.allclose(a.g[mir][:, :, ::-1], b.g, rtol=1e-11, atol=1e-13)


def test_transpose_symmetry():
    """On a square periodic grid, swapping x and y maps the solution onto its transpose: this catches
    a term that differs between the x and y components."""
    n = 20
    p = _params(n, n, lambda_mode="rho_cv_chi", chi=0.06)
    rho, T = _fields(n, n)
    a = model.run(p, model.init_state(p, rho, T), 30)
    b = model.run(p, model.init_state(p, rho.T.copy(), T.T.copy()), 30)
    tr = [0, 2, 1, 4, 3, 5, 8, 7, 6]
    assert np.allclose(a.f[tr].transpose(0, 2, 1), b.f, rtol=1e-11, atol=1e-13)
    assert np.allclose(a.g[tr].transpose(0, 2, 1), b.g, rtol=1e-11, atol=1e-13)


def test_nonphysical_state_is_reported():
    p = _params(8, 8)
    rho = np.full((8, 8), 1.0)
    rho[3, 5] = 11.0  # beyond the EOS pole 1/b = 10.5
    s = model.init_state(p, rho, np.full((8, 8), TS))
    with pytest.raises(model.OracleNonPhysical) as e:
        model.step(p, s)
    assert (e.value.x, e.value.y) == (5, 3)
