"""Checkpoint / resume (lbpc_save, lbpc_load): a run restored from a checkpoint taken after k steps
continues bit for bit like the uninterrupted run, in every precision and on both kernel paths, with
buoyancy (the lagged rho_ave is part of the state) and with the first-step source rule (phi_prev)."""

import numpy as np
import pytest

from paper_1709_04400_gb300 import lbpc, workloads

from .helpers import RL, RV, TC

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    from paper_1709_04400_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _run(case, rho, T, prec, path, steps):
    sim = lbpc.Simulation(lbpc.params_from_case(case, prec))
    sim.set_path(path)
    sim.init(rho, T)
    sim.step(steps)
    return sim


CASES = [(lbpc.FP64, lbpc.PATH_SPLIT), (lbpc.DF64, lbpc.PATH_SPLIT), (lbpc.FP32, lbpc.PATH_FUSED),
         (lbpc.FP16DEV, lbpc.PATH_FUSED), (lbpc.FP64, lbpc.PATH_FUSED)]
IDS = ["fp64-split", "df64-split", "fp32-fused", "fp16-fused", "fp64-fused"]


@pytest.mark.parametrize("prec,path", CASES, ids=IDS)
@pytest.mark.parametrize("k", [0, 7])
def test_resume_is_bitwise(prec, path, k):
    case, rho, T = workloads.mixed_small(TC, RV, RL, nx=45, ny=37)  # buoyancy, walls, strip, pressure top
    n = 20
    whole = _run(case, rho, T, prec, path, n)
    ref = whole.fields()
    whole.close()
    first = _run(case, rho, T, prec, path, k)
    ck = first.save()
    assert ck.size == first.checkpoint_bytes()
    first.close()
    second = lbpc.Simulation(lbpc.params_from_case(case, prec))
    second.set_path(path)
    second.load(ck)
    assert second.step_count == k
    second.step(n - k)
    got = second.fields()
    second.close()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_device_buffer_and_parameter_mismatch():
    import torch

    case, rho, T = workloads.mixed_small(TC, RV, RL, nx=33, ny=17)
    sim = _run(case, rho, T, lbpc.FP64, lbpc.PATH_AUTO, 5)
    buf = torch.empty(sim.checkpoint_bytes(), dtype=torch.uint8, device="cuda")
    sim.save(buf)
    ref_sim = _run(case, rho, T, lbpc.FP64, lbpc.PATH_AUTO, 9)
    ref = ref_sim.fields()
    ref_sim.close()
    sim.step(3)  # move on, then roll back to step 5 from the device copy
    sim.load(buf)
    sim.step(4)
    for a, b in zip(sim.fields(), ref):
        assert np.array_equal(a, b)
    other = lbpc.Simulation(lbpc.params_from_case(dict(case, cV=case["cV"] * 1.5), lbpc.FP64))
    with pytest.raises(lbpc.LbpcError) as e:
        other.load(buf)
    assert e.value.status == lbpc.LBPC_EINVAL
    other.close()
    bad = sim.save()
    bad[:8] = 0
    fresh = lbpc.Simulation(lbpc.params_from_case(case, lbpc.FP64))
    with pytest.raises(lbpc.LbpcError):
        fresh.load(bad)
    fresh.close()
    sim.close()
