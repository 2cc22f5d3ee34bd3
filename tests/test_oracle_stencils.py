"""Pins of the oracle's isotropic difference stencils (READING of the cited Eqs. (73)-(74)).

For a Fourier mode X = sin(kx x + ky y + c) the stencils have closed forms:
  d_x X  = sin(kx) (2 + cos ky)/3 * cos(...)
  lap X  = [ (4/3)(cos kx + cos ky - 2) + (2/3)(cos kx cos ky - 1) ] * X
which reduce to the exact derivatives kx cos(...) and -(kx^2 + ky^2) X as k -> 0.
"""

import numpy as np
import pytest

from oracle import model


def _p(nx, ny, ybc="periodic"):
    fb = ("periodic", "periodic", ybc, ybc)
    return model.OracleParams(nx=nx, ny=ny, flow_bc=fb)


@pytest.mark.parametrize("mx,my", [(1, 0), (2, 3), (5, 1), (7, 7)])
def test_fourier_symbols(mx, my):
    nx, ny = 48, 40
    kx, ky = 2 * np.pi * mx / nx, 2 * np.pi * my / ny
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    ph = kx * x + ky * y + 0.3
    X = np.sin(ph)
    p = _p(nx, ny)
    gx, gy = model.grad(X, p)
    assert np.allclose(gx, np.sin(kx) * (2 + np.cos(ky)) / 3 * np.cos(ph), atol=1e-14)
    assert np.allclose(gy, np.sin(ky) * (2 + np.cos(kx)) / 3 * np.cos(ph), atol=1e-14)
    lap = model.laplacian(X, p)
    sym = 4 / 3 * (np.cos(kx) + np.cos(ky) - 2) + 2 / 3 * (np.cos(kx) * np.cos(ky) - 1)
    assert np.allclose(lap, sym * X, atol=1e-14)


def test_second_order_convergence():
    errs = []
    for n in (16, 32, 64):
        k = 2 * np.pi / n
        y, x = np.mgrid[0:n, 0:n].astype(float)
        X = np.sin(k * x + 2 * k * y)
        lap = model.laplacian(X, _p(n, n))
        errs.append(np.abs(lap - (-(5 * k * k)) * X).max() / (5 * k * k))
    assert 3.7 < errs[0] / errs[1] < 4.3 and 3.7 < errs[1] / errs[2] < 4.3


def test_ghost_rows_copy_edge():
    """READING: a non-periodic y edge extends fields by copying the edge row. A field linear in y
    then has exact gradient 1 inside and 1/2 on the edge rows, and Laplacian -1/ +1 on them."""
    nx, ny = 8, 10
    y = np.arange(ny, dtype=float)[:, None] * np.ones((1, nx))
    p = _p(nx, ny, "wall")
    gx, gy = model.grad(y, p)
    assert np.allclose(gx, 0)
    assert np.allclose(gy[1:-1], 1.0) and np.allclose(gy[0], 0.5) and np.allclose(gy[-1], 0.5)
    lap = model.laplacian(y, p)
    assert np.allclose(lap[1:-1], 0.0, atol=1e-14)
    assert np.allclose(lap[0], 1.0) and np.allclose(lap[-1], -1.0)
