"""Which reference the binary16 deviation storage needs, measured on the FP64 oracle.

The library's FP16 storage keeps each post-collision population as a binary16 deviation from w_a * ref,
where ref is the storing node's own zeroth moment (density for f, T + S0 for g), kept in FP32 planes. A
reference shared by a whole instance (its mean) or by a 32 x 8 tile would drop those planes (80 instead
of 96 bytes per node and step). This test emulates the three formats on the oracle: after every
collision it rounds the deviations to binary16, then streams (the populations the step stores and the
next step pulls, Eq. 47). It compares the fields with the unrounded oracle after 1000 steps of the 64^2
evaporating droplet (R = 14, superheat 0.3 T_c), where liquid and vapour densities differ 17-fold.

Measured here (and, for the node reference, on the GPU: `test_gpu_evaporation_rate.py`):
- node reference: rho 5.2e-4, u 1.7e-2;
- tile reference: rho 6.5e-2, u 1.5;
- instance reference: rho 4.9e-2, u 0.35.
So a shared reference is about a hundred times worse, and the per-node planes stay."""

import numpy as np

from oracle import lattice as L
from oracle import model
from paper_1709_04400_gb300 import workloads

from .helpers import RL, RV, TC, max_rel, norm_rel, oracle_params

STEPS = 1000


def _rest_weights(p):
    """w_a of f (rest equilibrium of unit density) and of g (unit temperature), from the oracle."""
    one, zero = np.ones((1, 1)), np.zeros((1, 1))
    wf = L.from_moments(model.flow_meq(one, zero, zero))[:, 0, 0]
    wg = L.from_moments(model.heat_meq(one, zero, zero, p.model))[:, 0, 0]
    return wf, wg


def _reference(pop, kind):
    zeroth = pop.sum(axis=0)
    if kind == "node":
        return zeroth.astype(np.float32).astype(np.float64)  # the FP32 reference planes
    if kind == "instance":
        return np.full_like(zeroth, zeroth.mean())
    out = np.empty_like(zeroth)  # one mean per 32 x 8 tile
    ny, nx = zeroth.shape
    for y0 in range(0, ny, 8):
        for x0 in range(0, nx, 32):
            out[y0:y0 + 8, x0:x0 + 32] = zeroth[y0:y0 + 8, x0:x0 + 32].mean()
    return out


def _stored(pop, w, kind):
    base = w[:, None, None] * _reference(pop, kind)[None]
    return base + (pop - base).astype(np.float16).astype(np.float64)


def _step(p, s, kind, wf, wg):
    """model.step with the post-collision populations rounded to the storage format (improved model)."""
    mac = model.macroscopic(p, s)
    phi = mac["phi"]
    phi_prev = phi if s.phi_prev is None else s.phi_prev
    S0 = phi + 0.5 * (phi - phi_prev)
    fc = model.collide_flow(p, s.f, mac)
    gc = model.collide_heat(p, s.g, mac, S0)
    if kind is not None:
        fc, gc = _stored(fc, wf, kind), _stored(gc, wg, kind)
    fn = model.flow_boundaries(p, model.stream(fc), (mac["Fx"], mac["Fy"]))
    gn = model.heat_boundaries(p, model.stream(gc))
    return model.OracleState(f=fn, g=gn, phi_prev=phi, rho_ave=float(np.mean(mac["rho"])), step=s.step + 1,
                             last=mac)


def _fields_after(kind):
    case, rho, T = workloads.droplet_evaporation(TC, RV, RL, n=64, radius=14.0, dT_ratio=0.3)
    p = oracle_params(case)
    assert p.model == "improved"
    wf, wg = _rest_weights(p)
    s = model.init_state(p, rho, T)
    for _ in range(STEPS):
        s = _step(p, s, kind, wf, wg)
    return model.fields(p, s)


def test_unrounded_emulation_is_the_oracle_step():
    case, rho, T = workloads.droplet_evaporation(TC, RV, RL, n=64, radius=14.0, dT_ratio=0.3)
    p = oracle_params(case)
    wf, wg = _rest_weights(p)
    assert np.allclose(wf.sum(), 1.0) and np.allclose(wg.sum(), 1.0)
    a = b = model.init_state(p, rho, T)
    for _ in range(3):
        a, b = model.step(p, a), _step(p, b, None, wf, wg)
    assert np.array_equal(a.f, b.f) and np.array_equal(a.g, b.g)


def test_per_node_reference_is_needed():
    exact = _fields_after(None)

    def err(kind):
        got = _fields_after(kind)
        return dict(rho=max_rel(got[0], exact[0]), T=max_rel(got[3], exact[3]),
                    u=max(norm_rel(got[1], exact[1]), norm_rel(got[2], exact[2])))

    node, tile, inst = err("node"), err("tile"), err("instance")
    print(f"binary16 deviations after {STEPS} steps: node {node}, tile {tile}, instance {inst}")
    assert node["rho"] < 2e-3 and node["T"] < 2e-4 and node["u"] < 5e-2
    for shared in (tile, inst):
        assert shared["rho"] > 10 * node["rho"] and shared["u"] > 10 * node["u"]
