"""Seeded synthetic inputs shared by the GPU path and the oracle.

This module holds random-number generation and the geometry of the initial fields only; it
holds none of the lattice Boltzmann method's arithmetic (no equation of state, no moments, no
collision). Physical constants that depend on the method (coexistence densities, T_c) are
arguments supplied by the caller.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the two xor-shift-multiply rounds
and a final xor-shift; a double in [0, 1) is the top 53 bits times 2^-53.

Workloads (lattice units; Sec. IV of Li, Zhou & Yan for the physical set-ups):
  * droplet_periodic: the 128 x 128 periodic droplet (radius 25, tanh width 4) with a seeded
    sinusoidal temperature mode of amplitude 0.01 T_c about 0.86 T_c.
  * droplet_evaporation: an R = 40 droplet at the saturation temperature on 256 x 256, the outer
    ring held at T_s + dT (Sec. IV A's D^2-law case, resized).
  * heated_wall: 300 x 400 pool, liquid below y = ny/2, vapour above, uniform density noise
    +-1e-4, heated strip 20 nodes wide on the bottom wall (Sec. IV B's nucleation case, resized).
"""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 170904400


def splitmix64(seed, n):
    """n consecutive SplitMix64 outputs (uint64) from the given seed."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + _GOLDEN * np.arange(1, n + 1, dtype=np.uint64)
        z = state
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed, n):
    """n doubles in [0, 1) from SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def tanh_droplet(nx, ny, radius, width, rho_in, rho_out, cx=None, cy=None):
    """rho(r) = (rho_in + rho_out)/2 - (rho_in - rho_out)/2 tanh(2 (r - R)/W), row-major [ny][nx]."""
    cx = nx / 2.0 if cx is None else cx
    cy = ny / 2.0 if cy is None else cy
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    return 0.5 * (rho_in + rho_out) - 0.5 * (rho_in - rho_out) * np.tanh(2.0 * (r - radius) / width)


def tanh_layer(nx, ny, y_interface, width, rho_below, rho_above):
    """A flat interface at y = y_interface: rho_below under it, rho_above over it."""
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    return 0.5 * (rho_below + rho_above) - 0.5 * (rho_below - rho_above) * np.tanh(2.0 * (y - y_interface) / width)


def droplet_periodic(seed, nx, ny, radius, width, rho_l, rho_v, Tc, T_ratio=0.86, amp_ratio=0.01):
    """Droplet on a periodic grid with T = T_ratio T_c + amp_ratio T_c sin(2 pi (kx x/nx + ky y/ny) + theta).

    kx, ky in {1..4} and theta in [0, 2 pi) are drawn from the seed.
    """
    u = uniform(seed, 3)
    kx, ky = 1 + int(u[0] * 4), 1 + int(u[1] * 4)
    theta = 2.0 * np.pi * u[2]
    rho = tanh_droplet(nx, ny, radius, width, rho_l, rho_v)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    T = T_ratio * Tc + amp_ratio * Tc * np.sin(2.0 * np.pi * (kx * x / nx + ky * y / ny) + theta)
    return rho, T, dict(kx=kx, ky=ky, theta=theta)


def droplet_hot_ring(nx, ny, radius, width, rho_l, rho_v, T_sat, dT):
    """D^2-law start: tanh droplet at T_sat, vapour at T_sat + dT with the same tanh profile."""
    rho = tanh_droplet(nx, ny, radius, width, rho_l, rho_v)
    s = (rho_l - rho) / (rho_l - rho_v)  # 0 in the liquid, 1 in the vapour
    return rho, T_sat + dT * s


def pool_with_noise(seed, nx, ny, width, rho_l, rho_v, T_sat, amp=1e-4, surface=None):
    """Liquid below y = surface (default ny/2), vapour above, plus seeded uniform density noise in
    [-amp, amp)."""
    rho = tanh_layer(nx, ny, ny / 2.0 if surface is None else float(surface), width, rho_l, rho_v)
    rho = rho + amp * (2.0 * uniform(seed, nx * ny).reshape(ny, nx) - 1.0)
    return rho, np.full((ny, nx), T_sat)


def random_fields(seed, nx, ny, rho_l, rho_v, T0, dT):
    """Smooth but asymmetric random start used by small parity cases: a few seeded Fourier modes
    in rho (kept between rho_v and rho_l) and in T."""
    u = uniform(seed, 24)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    s = np.zeros((ny, nx))
    t = np.zeros((ny, nx))
    for k in range(4):
        kx, ky = 1 + int(u[6 * k] * 3), int(u[6 * k + 1] * 3)
        ph = 2 * np.pi * u[6 * k + 2]
        s += (0.5 + u[6 * k + 3]) * np.sin(2 * np.pi * (kx * x / nx + ky * y / ny) + ph)
        t += (0.5 + u[6 * k + 4]) * np.cos(2 * np.pi * (ky * x / nx + kx * y / ny) + 2 * np.pi * u[6 * k + 5])
    s = (s - s.min()) / (s.max() - s.min())
    t = (t - t.min()) / (t.max() - t.min())
    rho = rho_v + (rho_l - rho_v) * s
    return rho, T0 + dT * (t - 0.5)
