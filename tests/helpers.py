"""Shared test helpers: EOS constants from the oracle, case conversion and the parity metrics."""

import numpy as np

from oracle import eos, model

A, B, R, OM = 3.0 / 49.0, 2.0 / 21.0, 1.0, 0.344
TC = eos.critical_temperature(A, B, R)
TS = 0.86 * TC
RV, RL, PSAT = eos.maxwell_coexistence(TS, A, B, R, OM)

_ORACLE_KEYS = set(model.OracleParams.__dataclass_fields__)


def oracle_params(case: dict) -> model.OracleParams:
    return model.OracleParams(**{k: v for k, v in case.items() if k in _ORACLE_KEYS})


def run_oracle(case, rho, T, steps):
    p = oracle_params(case)
    s = model.run(p, model.init_state(p, rho, T), steps)
    return p, s


def max_rel(a, b):
    """max_i |a_i - b_i| / |b_i| (rho and T are bounded away from zero)."""
    return float(np.max(np.abs(a - b) / np.abs(b)))


def norm_rel(a, b):
    """||a - b||_inf / ||b||_inf (for u, which vanishes pointwise)."""
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def departed_bubble(rho, surface, min_area=10):
    """Area of the largest vapour region (rho below the mean of the coexistence densities, 4-connected)
    in the rows under surface - 15 that no longer touches the wall row; 0 while every such region is
    attached to the wall (or smaller than min_area)."""
    from scipy import ndimage

    r = np.asarray(rho)[: surface - 15]
    lab, n = ndimage.label(r < 0.5 * (RL + RV))
    best = 0
    for j in range(1, n + 1):
        ys = np.nonzero(lab == j)[0]
        if ys.min() > 0 and len(ys) >= min_area:
            best = max(best, len(ys))
    return best


def contact_angle(rho):
    """Contact angle of a droplet sitting on the y = 0 wall at the centre column, in degrees, from its
    height h and base half-width a (rho = (rho_l + rho_v)/2 located by linear interpolation along the
    centre column and along row 1): a circular cap has tan(theta/2) = h/a."""
    rho = np.asarray(rho)
    mid = 0.5 * (RL + RV)
    col = rho[:, rho.shape[1] // 2]
    j = int(np.nonzero(col > mid)[0].max())
    h = j + (col[j] - mid) / (col[j] - col[j + 1])
    row = rho[1]
    xs = np.nonzero(row > mid)[0]
    i0, i1 = int(xs.min()), int(xs.max())
    left = i0 - (row[i0] - mid) / (row[i0] - row[i0 - 1])
    right = i1 + (row[i1] - mid) / (row[i1] - row[i1 + 1])
    return float(np.degrees(2.0 * np.arctan(h / (0.5 * (right - left)))))


def poison_byte_buffers(monkeypatch):
    """Make torch.empty fill every uint8 buffer with 0xFF bytes: NaN in binary16, binary32 and binary64.
    Context workspaces and batch arenas are uint8 buffers, so a kernel that reads a byte the library
    never wrote turns its result into NaN."""
    import torch

    real_empty = torch.empty

    def empty(*args, **kwargs):
        t = real_empty(*args, **kwargs)
        if kwargs.get("dtype") == torch.uint8:
            t.fill_(255)
        return t

    monkeypatch.setattr(torch, "empty", empty)
