"""lbpc_step_static: the time step for callers that cannot allocate device memory.

Some callers have no way to hand the library a workspace (their device memory belongs to a pool
allocator they cannot extend, or cudaMalloc is not allowed where they run). For them
lbpc_step_static takes only the state and keeps its scratch in a static device array of the library.
This test calls it through the C ABI for two steps in a row. The result must match what the
ordinary entry point (lbpc_create + lbpc_step) produces from the same start, within the parity
tolerance the other FP64 tests use. The file is named to be collected last.
"""

import ctypes

import numpy as np
import pytest

from paper_1709_04400_gb300 import lbpc, workloads

from .helpers import RL, RV, TC

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _align256(n):
    return (n + 255) // 256 * 256


def test_static_step_matches_workspace_step():
    import torch

    from paper_1709_04400_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    lib = lbpc.load_library()
    case, rho, T = workloads.mixed_small(TC, RV, RL)  # walls, strip, pressure top, buoyancy
    params = lbpc.params_from_case(case, lbpc.FP64)
    N = params.nx * params.ny

    # the ordinary path: a context over a caller-owned workspace
    sim = lbpc.Simulation(params)
    sim.set_path(lbpc.PATH_SPLIT)
    sim.init(rho, T)
    mass0, _ = sim.sums()
    # A fresh context holds its state at the start of the workspace: post-collision f, then g, each
    # 9 N doubles rounded up to 256 bytes. Copy it into buffers this test owns.
    pop = _align256(9 * N * 8)
    ws = sim.workspace
    f_a = ws[0:9 * N * 8].view(torch.float64).clone()
    g_a = ws[pop:pop + 9 * N * 8].view(torch.float64).clone()
    f_b = torch.empty_like(f_a)
    g_b = torch.empty_like(g_a)
    # wall-row forces of the previous step (none before the first): [4][nx], A/B like the populations
    wall_a = torch.zeros(4 * params.nx, dtype=torch.float64, device="cuda")
    wall_b = torch.empty_like(wall_a)
    phi = torch.zeros(N, dtype=torch.float64, device="cuda")
    rho_ave = torch.tensor([mass0 / N], dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()

    c = params.to_c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def ptr(t):
        return ctypes.c_void_p(t.data_ptr())

    def static_step(fi, gi, wi, fo, go, wo, k):
        return lib.lbpc_step_static(ctypes.byref(c), ptr(fi), ptr(gi), ptr(fo), ptr(go), ptr(wi), ptr(wo), ptr(phi),
                                    ptr(rho_ave), k, stream)

    # two calls in a row: A -> B, then B -> A
    assert static_step(f_a, g_a, wall_a, f_b, g_b, wall_b, 0) == lbpc.LBPC_OK
    assert static_step(f_b, g_b, wall_b, f_a, g_a, wall_a, 1) == lbpc.LBPC_OK

    sim.step(2)  # the existing entry point from the same start; its state is back in the first half
    torch.cuda.synchronize()
    f_ref = ws[0:9 * N * 8].view(torch.float64).cpu().numpy()
    g_ref = ws[pop:pop + 9 * N * 8].view(torch.float64).cpu().numpy()
    f_st, g_st = f_a.cpu().numpy(), g_a.cpu().numpy()
    assert np.max(np.abs(f_st - f_ref)) / np.max(np.abs(f_ref)) < TOL
    assert np.max(np.abs(g_st - g_ref)) / np.max(np.abs(g_ref)) < TOL
    sim.close()


def test_static_step_rejects_grids_beyond_its_scratch():
    import torch

    lib = lbpc.load_library()
    big = lbpc.Params(nx=257, ny=256)  # one column beyond LBPC_STATIC_MAX_NODES = 256 * 256
    c = big.to_c()
    buf = torch.empty(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    s = lib.lbpc_step_static(ctypes.byref(c), p, p, p, p, p, p, p, p, 0, ctypes.c_void_p(0))
    assert s == lbpc.LBPC_ENOMEM
