"""Evaporation rate of a droplet against the FP64 oracle, for every precision and for instances advanced
inside a batch (the derived observable of the D^2 case, Sec. IV A).

The rate is the slope of the droplet area (workloads.droplet_area) fitted over steps 1000..4000 of a
64^2 droplet (R = 14, superheat 0.3 T_c), where the area falls linearly by about 9 %. Bars: 1 % for
the FP32 paths, alone and batched with other instances; 1e-6 for FP64 and DF64; the binary16
deviation storage is held to 5 % (its per-step population error is about 3e-4)."""

import numpy as np
import pytest

from paper_1709_04400_gb300 import lbpc, workloads

from .helpers import RL, RV, TC, max_rel, norm_rel, oracle_params

pytestmark = pytest.mark.gpu

STEPS, EVERY, FIT_FROM = 4000, 250, 1000


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    from paper_1709_04400_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _case():
    return workloads.droplet_evaporation(TC, RV, RL, n=64, radius=14.0, dT_ratio=0.3)


def _rate(hist):
    t = np.array([k for k, _ in hist], dtype=float)
    a = np.array([v for _, v in hist])
    sel = t >= FIT_FROM
    return np.polyfit(t[sel], a[sel], 1)[0]


_ORACLE_END = {}


@pytest.fixture(scope="module")
def oracle_rate():
    from oracle import model

    case, rho, T = _case()
    p = oracle_params(case)
    s = model.init_state(p, rho, T)
    hist = []
    for k in range(1, STEPS + 1):
        s = model.step(p, s)
        if k % EVERY == 0:
            hist.append((k, workloads.droplet_area(model.fields(p, s)[0])))
    _ORACLE_END["fields"] = model.fields(p, s)
    return _rate(hist)


# field errors after the 4000 steps, against the oracle's final fields (max relative for rho and T,
# relative to the largest |u| for the velocity)
FIELD_BARS = {lbpc.FP64: 1e-10, lbpc.DF64: 1e-10, lbpc.FP32: 1e-4, lbpc.FP16DEV: 5e-2}


def _field_errors(got):
    ref = _ORACLE_END["fields"]
    return dict(rho=max_rel(got[0], ref[0]), T=max_rel(got[3], ref[3]),
                u=max(norm_rel(got[1], ref[1]), norm_rel(got[2], ref[2])))


def _sim_rate(prec, path=lbpc.PATH_AUTO):
    case, rho, T = _case()
    sim = lbpc.Simulation(lbpc.params_from_case(case, prec))
    sim.set_path(path)
    sim.init(rho, T)
    hist = []
    for k in range(EVERY, STEPS + 1, EVERY):
        sim.step(EVERY)
        hist.append((k, workloads.droplet_area(sim.fields()[0])))
    end = sim.fields()
    sim.close()
    return _rate(hist), end


def _batch_rate(prec):
    """The droplet advanced inside a batch beside two other instances of other sizes and set-ups."""
    case, rho, T = _case()
    others = [workloads.droplet_evaporation(TC, RV, RL, n=96, radius=20.0, dT_ratio=0.1),
              workloads.mixed_small(TC, RV, RL, nx=37, ny=29)]
    ps = [lbpc.params_from_case(c, prec) for c, _, _ in [(case, rho, T)] + others]
    b = lbpc.Batch(prec, sum(lbpc.Batch.instance_bytes(p) for p in ps) + (64 << 20))
    i = b.add(ps[0], rho, T)
    for p, (_, r, t) in zip(ps[1:], others):
        b.add(p, r, t)
    hist = []
    for k in range(EVERY, STEPS + 1, EVERY):
        b.step(EVERY)
        hist.append((k, workloads.droplet_area(b.fields(i)[0])))
    end = b.fields(i)
    b.close()
    return _rate(hist), end


@pytest.mark.parametrize("prec,path,tol", [(lbpc.FP64, lbpc.PATH_SPLIT, 1e-6), (lbpc.DF64, lbpc.PATH_SPLIT, 1e-6),
                                           (lbpc.FP32, lbpc.PATH_FUSED, 1e-2), (lbpc.FP16DEV, lbpc.PATH_FUSED, 5e-2)],
                         ids=["fp64", "df64", "fp32", "fp16"])
def test_evaporation_rate_alone(oracle_rate, prec, path, tol):
    r, end = _sim_rate(prec, path)
    err = abs(r - oracle_rate) / abs(oracle_rate)
    fe = _field_errors(end)
    print(f"evaporation rate, prec {prec}: {r:.6e} per step against {oracle_rate:.6e} (relative error {err:.2e}); "
          f"fields after {STEPS} steps {fe}")
    assert oracle_rate < 0 and err <= tol
    assert all(v <= FIELD_BARS[prec] for v in fe.values()), fe


@pytest.mark.parametrize("prec,tol", [(lbpc.FP32, 1e-2), (lbpc.FP16DEV, 5e-2)], ids=["fp32", "fp16"])
def test_evaporation_rate_batched(oracle_rate, prec, tol):
    r, end = _batch_rate(prec)
    err = abs(r - oracle_rate) / abs(oracle_rate)
    fe = _field_errors(end)
    print(f"evaporation rate, batched prec {prec}: {r:.6e} per step against {oracle_rate:.6e} "
          f"(relative error {err:.2e}); fields after {STEPS} steps {fe}")
    assert err <= tol
    assert all(v <= FIELD_BARS[prec] for v in fe.values()), fe
