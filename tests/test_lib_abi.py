"""CPU checks of the C-ABI library: it builds, loads, exports every symbol include/lbpc.h declares,
and its host-side helpers (parameter validation, workspace sizing, EOS) behave. No GPU needed."""

import ctypes
import os
import re

import numpy as np
import pytest

from paper_1709_04400_gb300 import build, lbpc

from .helpers import RL, RV, TC, TS

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbpc.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "lbpc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbpc_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbpc.EXPORTED) == sorted(n for n in names)
    assert lib.lbpc_version() == 1


def test_struct_layout_matches_header():
    # 16 int32 then 39 doubles: no padding, 376 bytes
    assert ctypes.sizeof(lbpc.CParams) == 16 * 4 + (5 + 9 + 9 + 4 + 2 + 4 + 4 + 2) * 8
    assert lbpc.CParams.a.offset == 64


def test_check_params(lib):
    ok = lbpc.Params(nx=32, ny=16)
    assert lbpc.check_params(ok)[0] == lbpc.LBPC_OK
    bad = [
        dict(nx=1), dict(ny=0), dict(prec=7), dict(model=3),
        dict(flow_bc=(lbpc.WALL, lbpc.WALL, 0, 0)),
        dict(flow_bc=(0, 0, lbpc.WALL, 0)),
        dict(flow_bc=(0, 0, lbpc.WALL, lbpc.PRESSURE)),  # pressure edge needs rho_bc > 0
        dict(t_bc=(1, 0, 0, 0)),  # Dirichlet needs T_bc > 0
        dict(strip=(3, 9, 0.1)),  # strip needs a Dirichlet y- edge
        dict(s_g=(1.0,) * 8 + (2.0,)), dict(cV=0.0), dict(lam=-1.0), dict(b=0.0),
        dict(buoyancy=3), dict(buoyancy=-1),
        dict(buoyancy=2),  # the reference density of buoyancy 2 is held on a pressure y+ edge
        dict(buoyancy=2, flow_bc=(0, 0, lbpc.WALL, lbpc.WALL)),
    ]
    for kw in bad:
        p = lbpc.Params(**{**dict(nx=32, ny=16), **kw})
        s, msg = lbpc.check_params(p)
        assert s == lbpc.LBPC_EINVAL, (kw, msg)
        assert lbpc.workspace_bytes(p) == 0
    p = lbpc.Params(nx=32, ny=16, flow_bc=(0, 0, lbpc.WALL, lbpc.PRESSURE), rho_bc=(0, 0, 0, 0.4),
                    t_bc=(0, 0, 1, 1), T_bc=(0, 0, 0.09, 0.09), strip=(10, 20, 0.12))
    assert lbpc.check_params(p)[0] == lbpc.LBPC_OK


def test_workspace_grows_with_grid(lib):
    w1 = lbpc.workspace_bytes(lbpc.Params(nx=64, ny=64))
    w2 = lbpc.workspace_bytes(lbpc.Params(nx=128, ny=128))
    w3 = lbpc.workspace_bytes(lbpc.Params(nx=128, ny=128, prec=lbpc.FP32))
    # FP64: 4 x 9 population planes + phi + 12 scratch planes = 49 planes of 8 bytes per node
    assert 49 * 8 * 128 * 128 <= w2 < 49 * 8 * 128 * 128 + 64 * 1024
    assert w2 > 3.9 * w1 and w3 < 0.55 * w2
    # double-word storage and arithmetic: 8 bytes per value like FP64
    assert lbpc.workspace_bytes(lbpc.Params(nx=128, ny=128, prec=lbpc.DF64)) == w2


def test_eos_helpers_match_oracle(lib):
    p = lbpc.Params(nx=8, ny=8)
    Tc, pc = lbpc.eos_critical(p)
    assert Tc == pytest.approx(TC, rel=1e-15)
    rv, rl, ps = lbpc.coexistence(p, TS)
    # equal fugacity (library) against equal area (oracle): two routes to the same coexistence
    assert rv == pytest.approx(RV, rel=1e-11) and rl == pytest.approx(RL, rel=1e-11)
    with pytest.raises(lbpc.LbpcError):
        lbpc.coexistence(p, 1.01 * Tc)


def test_simulation_refuses_without_gpu():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        lbpc.Simulation(lbpc.Params(nx=8, ny=8))


def test_binding_refuses_device_buffers_of_the_wrong_size():
    """The binding checks the sizes of tensors whose pointers it passes to the kernels (a short tensor
    would be read or written past its end on the device). The checks run before any library call, so a
    context-less object stands in for a Simulation here."""
    import torch

    sim = object.__new__(lbpc.Simulation)
    sim.nx, sim.ny = 8, 6
    with pytest.raises(ValueError):
        sim.init(torch.zeros(47, dtype=torch.float64), torch.zeros(48, dtype=torch.float64))
    with pytest.raises(ValueError):
        sim.init(torch.zeros(48, dtype=torch.float64), torch.zeros(48, dtype=torch.float64),
                 ux=torch.zeros(40, dtype=torch.float64))
    for bad in (torch.zeros(1, dtype=torch.float64), torch.zeros(2, dtype=torch.float32),
                torch.zeros(4, dtype=torch.float64)[::2]):
        with pytest.raises(ValueError):
            sim.sums_async(bad)


def _every_workload():
    from paper_1709_04400_gb300 import serve, workloads

    yield workloads.droplet_periodic(TC, RV, RL)
    yield workloads.droplet_evaporation(TC, RV, RL)
    yield workloads.droplet_evaporation(TC, RV, RL, n=4096, radius=0.2 * 4096)
    for top in ("pressure", "wall"):
        yield workloads.heated_wall(TC, RV, RL, top=top)
    yield workloads.bubble_departure(TC, RV, RL)
    for model in ("improved", "compromised", "gong_cheng"):
        yield workloads.droplet_on_surface(TC, RV, RL, model=model, wall_T_ratio=0.875)
        yield workloads.paper_d2_law(TC, RV, RL, model=model)
    yield workloads.droplet_on_surface(TC, RV, RL, lambda_mode="const")
    for nx, ny in ((37, 29), (2, 3), (2, 2048), (3, 2048)):
        yield workloads.mixed_small(TC, RV, RL, nx=nx, ny=ny)
    yield from workloads.batched_evaporation(TC, RV, RL, count=8)
    for req in serve.poisson_stream(40, 1.0, seed=11):
        yield serve.make_case(req, TC, RV, RL)


def test_every_workload_is_accepted_by_library_and_oracle(lib):
    """Each seeded workload (the bench's, the tests', the paper cases', the service's requests) passes
    the library's parameter check in every precision and the oracle's, and its initial fields have the
    grid's shape and physical values (0 < rho < 1/b, T > 0)."""
    from .helpers import oracle_params

    b = 2.0 / 21.0
    count = 0
    for case, rho, T in _every_workload():
        assert rho.shape == T.shape == (case["ny"], case["nx"]), case["name"]
        assert np.all(rho > 0) and np.all(rho < 1.0 / b) and np.all(T > 0), case["name"]
        oracle_params(case).check()
        for prec in (lbpc.FP64, lbpc.DF64, lbpc.FP32, lbpc.FP16DEV):
            s, msg = lbpc.check_params(lbpc.params_from_case(case, prec))
            assert s == lbpc.LBPC_OK, (case["name"], prec, msg)
        count += 1
    assert count > 60
