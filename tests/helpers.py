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
