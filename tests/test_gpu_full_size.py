"""Parity at the workloads' full sizes, in the launch configurations the bench times, on outputs the
oracle can compute.

- Large grids (4096^2 FP32 and FP16 deviation storage, 2048^2 FP64). After k steps, the result at a node
  depends only on the populations within 3k nodes of it: the pull reaches 1 node, the psi stencil of
  the force 1 more, and the velocity stencil of the source 1 more. A W x W window of the initial fields,
  stepped by the oracle with any boundary at its edge (periodic here), therefore reproduces the full
  grid's result on its central (W - 6k)^2 nodes. The window sits on the droplet interface, where the
  step does the most, far from the held-temperature ring at the domain edge.
- The batched workload (256 uneven instances, default and tuned configurations): the three smallest
  instances are compared with the oracle after the batch has advanced together, and windows of the three
  largest (sides of about 500) are compared in the same way as the large grids."""

import numpy as np
import pytest

from paper_1709_04400_gb300 import lbpc, workloads

from .helpers import RL, RV, TC, max_rel, norm_rel, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    from paper_1709_04400_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _window_check(n, prec, tol, tol_u, k=10, W=128):
    case, rho, T = workloads.droplet_evaporation(TC, RV, RL, n=n, radius=0.2 * n, dT_ratio=0.1)
    sim = lbpc.Simulation(lbpc.params_from_case(case, prec))
    sim.init(rho, T)
    sim.step(k)
    full = sim.fields()
    sim.close()
    # window centred on the interface, right of the droplet centre
    cx, cy = n // 2 + int(round(0.2 * n)), n // 2
    x0, y0 = cx - W // 2, cy - W // 2
    sl = (slice(y0, y0 + W), slice(x0, x0 + W))
    wcase = dict(case, name=f"window_{n}", nx=W, ny=W, t_bc=("none",) * 4, T_bc=(0.0,) * 4)
    p, s = run_oracle(wcase, rho[sl], T[sl], k)
    from oracle import model

    ref = model.fields(p, s)
    m = 3 * k
    inner = (slice(m, W - m), slice(m, W - m))
    got = [f[sl][inner] for f in full]
    exp = [f[inner] for f in ref]
    err = dict(rho=max_rel(got[0], exp[0]), T=max_rel(got[3], exp[3]), ux=norm_rel(got[1], exp[1]),
               uy=norm_rel(got[2], exp[2]))
    print(f"{n}^2 prec {prec}, window {W}^2 after {k} steps, central {W - 2 * m}^2: {err}")
    assert err["rho"] <= tol and err["T"] <= tol and err["ux"] <= tol_u and err["uy"] <= tol_u, err


# binary16 deviation storage keeps the documented bound of its own parity test: 1e-3 on rho and T,
# 2e-2 on u relative to the (small) velocities. Binary32: the field bar of 1e-4 on rho, T and u (u
# relative to the largest |u|, still small ten steps after a start from rest).
@pytest.mark.parametrize("n,prec,tol,tol_u", [(4096, lbpc.FP32, 1e-4, 1e-4), (4096, lbpc.FP16DEV, 1e-3, 2e-2),
                                              (2048, lbpc.FP64, 1e-10, 1e-10), (2048, lbpc.DF64, 1e-10, 1e-10)],
                         ids=["fp32-4096", "fp16-4096", "fp64-2048", "df64-2048"])
def test_large_grid_window(n, prec, tol, tol_u):
    _window_check(n, prec, tol, tol_u)


@pytest.mark.parametrize("tuned", [False, True], ids=["default", "tuned"])
def test_batched_full_size_sampled(tuned):
    insts = workloads.batched_evaporation(TC, RV, RL, count=256)
    ps = [lbpc.params_from_case(c, lbpc.FP32) for c, _, _ in insts]
    b = lbpc.Batch(lbpc.FP32, sum(lbpc.Batch.instance_bytes(p) for p in ps) + (256 << 20), max_instances=300)
    ids = [b.add(p, r, t) for p, (_, r, t) in zip(ps, insts)]
    steps = 40
    if tuned:
        b.autotune(steps_per_candidate=1)  # advances the batch by real steps
    start = b.step_count(ids[0])
    b.step(steps - start if start < steps else 0)
    n_done = b.step_count(ids[0])
    b.check()
    order = np.argsort([c["nx"] * c["ny"] for c, _, _ in insts])[:3]
    for j in order:
        case, rho, T = insts[j]
        got = b.fields(ids[j])
        p, s = run_oracle(case, rho, T, n_done)
        from oracle import model

        ref = model.fields(p, s)
        err = dict(rho=max_rel(got[0], ref[0]), T=max_rel(got[3], ref[3]), ux=norm_rel(got[1], ref[1]),
                   uy=norm_rel(got[2], ref[2]))
        print(f"batched instance {j} ({case['nx']}x{case['ny']}) after {n_done} steps: {err}")
        assert all(v <= 1e-4 for v in err.values()), (j, err)
    b.close()


@pytest.mark.parametrize("config", [None, (0, 128)], ids=["default", "variant0-128"])
def test_batched_largest_instances_windows(config):
    """The three largest of the 256 instances (sides of about 500), each compared with the oracle on a
    128^2 window after 10 steps of the whole batch (central 68^2 nodes), at the FP32 field bar. The window
    sits on the interface right of the droplet's centre, like the large-grid windows above, clear of the
    held-temperature ring."""
    insts = workloads.batched_evaporation(TC, RV, RL, count=256)
    ps = [lbpc.params_from_case(c, lbpc.FP32) for c, _, _ in insts]
    b = lbpc.Batch(lbpc.FP32, sum(lbpc.Batch.instance_bytes(p) for p in ps) + (256 << 20), max_instances=300)
    ids = [b.add(p, r, t) for p, (_, r, t) in zip(ps, insts)]
    if config is not None:
        b.set_config(*config)
    k, W = 10, 128
    b.step(k)
    b.check()
    from oracle import model

    largest = np.argsort([c["nx"] * c["ny"] for c, _, _ in insts])[-3:]
    for j in largest:
        case, rho, T = insts[j]
        n = case["nx"]
        assert n >= 480 and b.step_count(ids[j]) == k
        got_full = b.fields(ids[j])
        R = int(round(np.sqrt(np.count_nonzero(rho > 0.5 * (RL + RV)) / np.pi)))  # initial droplet radius
        x0, y0 = n // 2 + R - W // 2, n // 2 - W // 2
        assert x0 > 3 * k and x0 + W < n - 3 * k
        sl = (slice(y0, y0 + W), slice(x0, x0 + W))
        wcase = dict(case, name=f"window_{n}", nx=W, ny=W, t_bc=("none",) * 4, T_bc=(0.0,) * 4)
        p, s = run_oracle(wcase, rho[sl], T[sl], k)
        ref = model.fields(p, s)
        m = 3 * k
        inner = (slice(m, W - m), slice(m, W - m))
        got = [f[sl][inner] for f in got_full]
        exp = [f[inner] for f in ref]
        err = dict(rho=max_rel(got[0], exp[0]), T=max_rel(got[3], exp[3]), ux=norm_rel(got[1], exp[1]),
                   uy=norm_rel(got[2], exp[2]))
        print(f"batched instance {j} ({n}x{n}), window {W}^2 after {k} steps, central {W - 2 * m}^2: {err}")
        assert all(v <= 1e-4 for v in err.values()), (j, err)
    b.close()
