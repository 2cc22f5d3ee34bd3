"""D2Q9 lattice and MRT moment algebra (oracle; test infrastructure only).

Velocity ordering e0=(0,0), e1=(1,0), e2=(0,1), e3=(-1,0), e4=(0,-1), e5=(1,1), e6=(-1,1),
e7=(-1,-1), e8=(1,-1). Weights w0=4/9, w1-4=1/9, w5-8=1/36 (Sec. II B, after Eq. 14).
c = dx/dt = 1, c_s^2 = 1/3.

M is the orthogonal D2Q9 transformation matrix of the MRT operator (Eqs. 42-43) with rows
(rho, e, eps, jx, qx, jy, qy, pxx, pxy). The paper does not print M; READING: it is the
Lallemand-Luo matrix, the only row convention under which M g_eq(Eq. 29) equals Eq. 44, which the
tests check in exact rational arithmetic. Its rows are mutually orthogonal, so
M^{-1} = M^T diag(1 / |row_k|^2).
"""

from fractions import Fraction

import numpy as np

CS2 = 1.0 / 3.0

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=np.int64)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=np.int64)
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6], dtype=np.int64)

W_FRAC = [Fraction(4, 9)] + [Fraction(1, 9)] * 4 + [Fraction(1, 36)] * 4
W = np.array([float(x) for x in W_FRAC])

M_INT = np.array(
    [
        [1, 1, 1, 1, 1, 1, 1, 1, 1],  # rho (T for the thermal set)
        [-4, -1, -1, -1, -1, 2, 2, 2, 2],  # e
        [4, -2, -2, -2, -2, 1, 1, 1, 1],  # eps
        [0, 1, 0, -1, 0, 1, -1, -1, 1],  # jx
        [0, -2, 0, 2, 0, 1, -1, -1, 1],  # qx
        [0, 0, 1, 0, -1, 1, 1, -1, -1],  # jy
        [0, 0, -2, 0, 2, 1, 1, -1, -1],  # qy
        [0, 1, -1, 1, -1, 0, 0, 0, 0],  # pxx
        [0, 0, 0, 0, 0, 1, -1, 1, -1],  # pxy
    ],
    dtype=np.int64,
)


def m_inverse_fractions():
    """M^{-1} = M^T diag(1/|row_k|^2) as exact fractions (rows of M are orthogonal)."""
    norms = [sum(int(v) * int(v) for v in row) for row in M_INT]
    return [[Fraction(int(M_INT[k, a]), norms[k]) for k in range(9)] for a in range(9)]


M = M_INT.astype(np.float64)
MINV = np.array([[float(x) for x in row] for row in m_inverse_fractions()])


def to_moments(pop):
    """m = M g for a population array of shape (9, ...) (Eq. 42, 'm = Mg')."""
    return np.einsum("ka,a...->k...", M, pop)


def from_moments(mom):
    """g = M^{-1} m for a moment array of shape (9, ...) (Eq. 47, 'g* = M^{-1} m*')."""
    return np.einsum("ak,k...->a...", MINV, mom)
