"""lbpc_step_static: the time step for callers that cannot allocate device memory.

Some callers have no way to hand the library a workspace: their device memory belongs to a pool
allocator they cannot extend, or cudaMalloc is not allowed where they run. For them lbpc_step_static
takes only the state and keeps its scratch in a static device array of the library.

This test runs the ordinary entry point (lbpc_create + lbpc_step, split organisation) for two steps and
takes its state before and after from checkpoints (lbpc_save, whose layout include/lbpc.h documents).
It then calls lbpc_step_static through the C ABI twice in a row from the same start. The kernels are the
same, so the populations, phi and the wall-row forces must agree bit for bit, in every precision the
call accepts. The second call must leave the device's free memory unchanged. The file is named so that
pytest collects it last.
"""

import ctypes
import struct

import numpy as np
import pytest

from paper_1709_04400_gb300 import lbpc, workloads

from .helpers import RL, RV, TC

pytestmark = pytest.mark.gpu

HEADER = 512
STORE = {lbpc.FP64: 8, lbpc.FP32: 4, lbpc.DF64: 8}  # bytes per stored population
REAL = {lbpc.FP64: 8, lbpc.FP32: 4, lbpc.DF64: 8}  # bytes per value of the arithmetic type (phi)


def _sections(buf, prec, nx, ny):
    """f, g, phi, wall and rho_ave of a checkpoint (header: magic, version, header size, lbpc_params,
    step, rho_ave, section sizes; then f, g, phi, wall for storage without reference planes)."""
    N = nx * ny
    assert bytes(buf[:8]) == b"LBPCCKP1"
    off = 16 + ctypes.sizeof(lbpc.CParams)
    step, rho_ave = struct.unpack_from("<qd", bytes(buf[off:off + 16]))
    pop = 9 * N * STORE[prec]
    o = HEADER
    f = buf[o:o + pop]
    g = buf[o + pop:o + 2 * pop]
    o += 2 * pop
    phi = buf[o:o + N * REAL[prec]]
    o += N * REAL[prec]
    wall = buf[o:o + 4 * nx * 8]
    return dict(f=f, g=g, phi=phi, wall=wall, step=step, rho_ave=rho_ave)


@pytest.mark.parametrize("prec", [lbpc.FP64, lbpc.FP32, lbpc.DF64], ids=["fp64", "fp32", "df64"])
def test_static_step_matches_workspace_step(prec):
    import torch

    from paper_1709_04400_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    lib = lbpc.load_library()
    case, rho, T = workloads.mixed_small(TC, RV, RL)  # walls, strip, pressure top, buoyancy
    params = lbpc.params_from_case(case, prec)
    nx, ny = params.nx, params.ny

    # the ordinary path: a context over a caller-owned workspace, checkpointed before and after two steps
    sim = lbpc.Simulation(params)
    sim.set_path(lbpc.PATH_SPLIT)
    sim.init(rho, T)
    start = _sections(sim.save(), prec, nx, ny)
    sim.step(2)
    ref = _sections(sim.save(), prec, nx, ny)
    sim.close()
    assert start["step"] == 0 and ref["step"] == 2

    dev = lambda a: torch.from_numpy(np.array(a, dtype=np.uint8)).cuda()  # noqa: E731
    f_a, g_a, wall_a = dev(start["f"]), dev(start["g"]), dev(start["wall"])
    f_b, g_b, wall_b = torch.empty_like(f_a), torch.empty_like(g_a), torch.empty_like(wall_a)
    phi = torch.zeros(nx * ny * REAL[prec], dtype=torch.uint8, device="cuda")  # ignored on input at step 0
    rho_ave = torch.tensor([start["rho_ave"]], dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()

    c = params.to_c()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def ptr(t):
        return ctypes.c_void_p(t.data_ptr())

    def static_step(fi, gi, wi, fo, go, wo, k):
        return lib.lbpc_step_static(ctypes.byref(c), ptr(fi), ptr(gi), ptr(fo), ptr(go), ptr(wi), ptr(wo), ptr(phi),
                                    ptr(rho_ave), k, stream)

    # two calls in a row: A -> B, then B -> A; the second must not touch the device's free memory
    assert static_step(f_a, g_a, wall_a, f_b, g_b, wall_b, 0) == lbpc.LBPC_OK
    free_before = torch.cuda.mem_get_info()[0]
    assert static_step(f_b, g_b, wall_b, f_a, g_a, wall_a, 1) == lbpc.LBPC_OK
    free_after = torch.cuda.mem_get_info()[0]
    assert free_after == free_before

    for name, got in (("f", f_a), ("g", g_a), ("phi", phi), ("wall", wall_a)):
        exp = np.frombuffer(bytes(ref[name]), dtype=np.uint8)
        assert np.array_equal(got.cpu().numpy(), exp), name
    assert rho_ave.item() == ref["rho_ave"]


def test_static_step_rejects_grids_beyond_its_scratch():
    import torch

    lib = lbpc.load_library()
    big = lbpc.Params(nx=257, ny=256)  # one column beyond LBPC_STATIC_MAX_NODES = 256 * 256
    c = big.to_c()
    buf = torch.empty(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    s = lib.lbpc_step_static(ctypes.byref(c), p, p, p, p, p, p, p, p, 0, ctypes.c_void_p(0))
    assert s == lbpc.LBPC_ENOMEM
