"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bar: FP64 storage and arithmetic within 1e-10 relative error on rho, u and T (max_i |a-b|/|b| for
rho and T, ||a-b||_inf/||b||_inf for u, which vanishes pointwise); FP32 within 1e-4 on the same
metrics. The double-word precision (LBPC_DF64: pairs of binary32, 48-bit significand) is held to the
FP64 bar. Grids are ragged (not multiples of the 256-thread block) and span many blocks."""

import numpy as np
import pytest

from oracle import model
from paper_1709_04400_gb300 import lbpc, workloads

from .helpers import RL, RV, TC, TS, max_rel, norm_rel, oracle_params, poison_byte_buffers, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    from paper_1709_04400_gb300 import build

    build.build()
    torch.cuda.set_device(0)


PATHS = [lbpc.PATH_SPLIT, lbpc.PATH_FUSED]
PATH_IDS = ["split", "fused"]
F64 = [lbpc.FP64, lbpc.DF64]  # precisions held to the FP64 bar
F64_IDS = ["fp64", "df64"]

_ORACLE = {}


def _oracle(key, case, rho, T, steps):
    """run_oracle, computed once per (key, steps) in this module."""
    if (key, steps) not in _ORACLE:
        _ORACLE[(key, steps)] = run_oracle(case, rho, T, steps)
    return _ORACLE[(key, steps)]


def _gpu(case, rho, T, steps, prec=lbpc.FP64, path=lbpc.PATH_AUTO):
    sim = lbpc.Simulation(lbpc.params_from_case(case, prec))
    sim.set_path(path)
    sim.init(rho, T)
    sim.step(steps)
    out = sim.fields()
    f, g = sim.populations()
    sums = sim.sums()
    sim.close()
    return out, f, g, sums


def _errors(gpu, p, s):
    r_o, ux_o, uy_o, T_o = model.fields(p, s)
    r_g, ux_g, uy_g, T_g = gpu
    return dict(rho=max_rel(r_g, r_o), T=max_rel(T_g, T_o), ux=norm_rel(ux_g, ux_o), uy=norm_rel(uy_g, uy_o))


def _assert_within(err, tol):
    bad = {k: v for k, v in err.items() if not v <= tol}
    assert not bad, f"errors above {tol}: {err}"


@pytest.mark.parametrize("prec", F64, ids=F64_IDS)
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_mixed_boundaries_fp64(path, prec):
    """Wall + strip + pressure top + buoyancy + lambda = rho c_V chi + distinct thermal rates."""
    case, rho, T = workloads.mixed_small(TC, RV, RL)
    steps = 150
    gpu, f, g, _ = _gpu(case, rho, T, steps, prec=prec, path=path)
    p, s = _oracle("mixed_small", case, rho, T, steps)
    _assert_within(_errors(gpu, p, s), 1e-10)
    assert np.max(np.abs(f - s.f)) / np.max(np.abs(s.f)) < 1e-10
    assert np.max(np.abs(g - s.g)) / np.max(np.abs(s.g)) < 1e-10


def _closed_wettable_pool():
    """Both y edges are walls with a wettable bottom (G_w = -0.2), buoyancy and a hot strip: the wall
    rows' force of the previous step enters the closure on both walls, the adsorption acts on the
    bottom wall only, and the lid stays neutral."""
    case, rho, T = workloads.mixed_small(TC, RV, RL, nx=45, ny=31)
    case = dict(case, name="closed_wettable_45x31", flow_bc=("periodic", "periodic", "wall", "wall"),
                rho_bc=(0.0,) * 4)
    return case, rho, T


@pytest.mark.parametrize("prec", F64, ids=F64_IDS)
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_closed_pool_wettable_walls_fp64(path, prec):
    case, rho, T = _closed_wettable_pool()
    steps = 200
    gpu, f, g, (mass, _) = _gpu(case, rho, T, steps, prec=prec, path=path)
    p, s = _oracle("closed_wettable", case, rho, T, steps)
    _assert_within(_errors(gpu, p, s), 1e-10)
    assert np.max(np.abs(f - s.f)) / np.max(np.abs(s.f)) < 1e-10
    assert abs(mass - s.f.sum()) / s.f.sum() < 1e-12


# FP32: the 1e-4 bar; binary16 deviation storage: its documented bounds (rho and T 1e-3 per 100 steps,
# u 2e-2 relative to the small velocities)
@pytest.mark.parametrize("prec,tol,tol_u", [(lbpc.FP32, 1e-4, 1e-4), (lbpc.FP16DEV, 2e-3, 2e-2)], ids=["fp32", "fp16"])
def test_closed_pool_wettable_walls_reduced(prec, tol, tol_u):
    case, rho, T = _closed_wettable_pool()
    gpu, *_ = _gpu(case, rho, T, 200, prec=prec, path=lbpc.PATH_FUSED)
    p, s = _oracle("closed_wettable", case, rho, T, 200)
    err = _errors(gpu, p, s)
    print(f"closed wettable pool, prec {prec}, 200 steps: {err}")
    assert err["rho"] <= tol and err["T"] <= tol and err["ux"] <= tol_u and err["uy"] <= tol_u, err


@pytest.mark.parametrize("prec", F64, ids=F64_IDS)
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("mdl", ["compromised", "gong_cheng"])
def test_comparison_models_fp64(path, mdl, prec):
    """The comparison models of Sec. IV: compromised (Eq. 44, no corrections) and Gong-Cheng (Eqs. 12-14)."""
    case, rho, T = workloads.mixed_small(TC, RV, RL, nx=33, ny=17)
    case = dict(case, model=mdl)
    gpu, *_ = _gpu(case, rho, T, 100, prec=prec, path=path)
    p, s = _oracle(("mixed_33x17", mdl), case, rho, T, 100)
    _assert_within(_errors(gpu, p, s), 1e-10)


@pytest.mark.parametrize("prec", F64, ids=F64_IDS)
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_wall_top_and_pressure_bottom_fp64(path, prec):
    """The mirrored boundary set: wall on y+, pressure on y-, adiabatic (no Dirichlet) top."""
    case, rho, T = workloads.mixed_small(TC, RV, RL, nx=19, ny=23)
    rho = rho[::-1].copy()
    case = dict(case, flow_bc=("periodic", "periodic", "pressure", "wall"), rho_bc=(0, 0, RV, 0),
                t_bc=("none", "none", "dirichlet", "none"), strip=None, gy=3e-5)
    gpu, *_ = _gpu(case, rho, T, 100, prec=prec, path=path)
    p, s = _oracle("mirrored_19x23", case, rho, T, 100)
    _assert_within(_errors(gpu, p, s), 1e-10)


@pytest.mark.parametrize("prec", F64, ids=F64_IDS)
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_droplet_periodic_128_fp64_1000_steps(path, prec):
    """The 128 x 128 periodic droplet: 1000 steps, 1e-10 on rho, u, T (the FP64 parity bar)."""
    case, rho, T = workloads.droplet_periodic(TC, RV, RL)
    gpu, _, _, (mass, heat) = _gpu(case, rho, T, 1000, prec=prec, path=path)
    p, s = _oracle("droplet_periodic_128", case, rho, T, 1000)
    err = _errors(gpu, p, s)
    print(f"droplet 128^2, 1000 steps, prec {prec}, path {path}: {err}")
    _assert_within(err, 1e-10)
    assert abs(mass - s.f.sum()) / s.f.sum() < 1e-12
    assert abs(heat - s.g.sum()) / s.g.sum() < 1e-12


@pytest.mark.parametrize("prec", F64, ids=F64_IDS)
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
@pytest.mark.parametrize("dT", [0.05, 0.1, 0.2])
def test_droplet_evaporation_256_fp64(dT, path, prec):
    """The 256 x 256 evaporation case at full size, 200 steps (the oracle's share of the run)."""
    case, rho, T = workloads.droplet_evaporation(TC, RV, RL, dT_ratio=dT)
    gpu, *_ = _gpu(case, rho, T, 200, prec=prec, path=path)
    p, s = _oracle(("evaporation_256", dT), case, rho, T, 200)
    err = _errors(gpu, p, s)
    print(f"evaporation 256^2 dT {dT}, 200 steps, prec {prec}, path {path}: {err}")
    _assert_within(err, 1e-10)


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_heated_wall_fp32(path):
    """The 300 x 400 heated-wall pool in FP32 storage and arithmetic against the FP64 oracle."""
    case, rho, T = workloads.heated_wall(TC, RV, RL)
    steps = 100
    gpu, *_ = _gpu(case, rho, T, steps, prec=lbpc.FP32, path=path)
    p, s = run_oracle(case, rho, T, steps)
    _assert_within(_errors(gpu, p, s), 1e-4)


def test_mass_conservation_gpu():
    """Mass is conserved to round-off: each step rounds every population once (relative 2^-53), so
    the drift after n steps stays below n * 5 * 1.1e-16."""
    case, rho, T = workloads.droplet_periodic(TC, RV, RL, n=64, radius=12.0)
    sim = lbpc.Simulation(lbpc.params_from_case(case))
    sim.init(rho, T)
    m0, _ = sim.sums()
    n = 2000
    sim.step(n)
    m1, _ = sim.sums()
    sim.close()
    assert abs(m1 - m0) / m0 < n * 5 * 1.1e-16


def test_smallest_grid_and_zero_steps():
    """2 x 3 nodes (the smallest grid with non-periodic y), vapour near saturation, every boundary class."""
    case, _, _ = workloads.mixed_small(TC, RV, RL, nx=2, ny=3)
    rho = RV * (1.0 + 0.01 * np.arange(6).reshape(3, 2))
    T = np.full((3, 2), TS)
    gpu, *_ = _gpu(case, rho, T, 0)
    p = oracle_params(case)
    s = model.init_state(p, rho, T)
    _assert_within(_errors(gpu, p, s), 1e-13)
    gpu, *_ = _gpu(case, rho, T, 5)
    s = model.run(p, s, 5)
    _assert_within(_errors(gpu, p, s), 1e-10)


@pytest.mark.parametrize("nx", [2, 3])
@pytest.mark.parametrize("prec,tol", [(lbpc.FP64, 1e-10), (lbpc.FP32, 1e-4)], ids=["fp64", "fp32"])
def test_narrow_tall_channel_fused(prec, tol, nx):
    """nx = 2 or 3, ny = 2048 with the domain-mean buoyancy on the fused path: 256 tiles of 32 x 8 for
    only 4096-6144 nodes, more tiles than 64-node blocks. Each tile's partial sum of rho must land in
    its own slot, and the mean they give must be the oracle's."""
    case, rho, T = workloads.mixed_small(TC, RV, RL, nx=nx, ny=2048)
    steps = 20
    p, s = _oracle(f"narrow_{nx}", case, rho, T, steps)
    gpu, _, _, _ = _gpu(case, rho, T, steps, prec=prec, path=lbpc.PATH_FUSED)
    _assert_within(_errors(gpu, p, s), tol)


def test_tall_channel_takes_the_split_step():
    """ny = 524,296 needs 65,537 rows of 32 x 8 tiles, more rows of CTAs than a launch holds: FP32 on
    the default path takes the split step (same bits as asking for it) and agrees with the oracle; asking
    for the fused step is refused and leaves the context usable."""
    case, rho, T = workloads.mixed_small(TC, RV, RL, nx=2, ny=524_296)
    steps = 3
    out = []
    for path in (lbpc.PATH_AUTO, lbpc.PATH_SPLIT):
        sim = lbpc.Simulation(lbpc.params_from_case(case, lbpc.FP32))
        if path == lbpc.PATH_AUTO:
            with pytest.raises(lbpc.LbpcError):
                sim.set_path(lbpc.PATH_FUSED)
        sim.set_path(path)
        sim.init(rho, T)
        sim.step(steps)
        out.append(sim.fields())
        sim.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    p, s = run_oracle(case, rho, T, steps)
    err = _errors(out[0], p, s)
    # the FP32 field bar on every field (u relative to the largest |u|, which is small three steps after
    # a start from rest)
    assert err["rho"] <= 1e-4 and err["T"] <= 1e-4 and err["ux"] <= 1e-4 and err["uy"] <= 1e-4, err


def test_device_pointers_and_async_steps():
    import torch

    case, rho, T = workloads.mixed_small(TC, RV, RL)
    sim = lbpc.Simulation(lbpc.params_from_case(case))
    sim.init(torch.from_numpy(rho).cuda(), torch.from_numpy(T).cuda())
    for _ in range(10):
        sim.step(3, sync=False)
    sim.check()
    assert sim.step_count == 30
    dev = [t.cpu().numpy() for t in sim.fields(device=True)]
    host = sim.fields()
    for a, b in zip(dev, host):
        assert np.array_equal(a, b)
    sim.close()
    p, s = run_oracle(case, rho, T, 30)
    _assert_within(_errors(host, p, s), 1e-10)


def test_nonphysical_state_reported():
    case, rho, T = workloads.droplet_periodic(TC, RV, RL, n=32, radius=8.0)
    rho = rho.copy()
    rho[7, 11] = 11.0  # beyond the EOS pole 1/b = 10.5
    sim = lbpc.Simulation(lbpc.params_from_case(case))
    sim.init(rho, T)
    with pytest.raises(lbpc.LbpcError) as e:
        sim.step(3)
    assert e.value.status == lbpc.LBPC_ENONPHYS
    assert "step 0, node (x=11, y=7)" in str(e.value)
    with pytest.raises(lbpc.LbpcError) as e2:
        sim.step(1)
    assert e2.value.status == lbpc.LBPC_ESTATE
    sim.fields()  # still readable
    sim.close()


def test_failure_matches_oracle():
    """A degenerate 2 x 3 pool (liquid under a vapour-density edge one node away) leaves the EOS range;
    the GPU reports the same first step and node as the oracle."""
    case, rho, T = workloads.mixed_small(TC, RV, RL, nx=2, ny=3)
    p = oracle_params(case)
    s = model.init_state(p, rho, T)
    with pytest.raises(model.OracleNonPhysical) as eo:
        model.run(p, s, 10)
    sim = lbpc.Simulation(lbpc.params_from_case(case))
    sim.init(rho, T)
    with pytest.raises(lbpc.LbpcError) as eg:
        sim.step(10)
    sim.close()
    assert eg.value.status == lbpc.LBPC_ENONPHYS
    assert f"step {eo.value.step}, node (x={eo.value.x}, y={eo.value.y})" in str(eg.value)


@pytest.mark.parametrize("prec,tol", [(lbpc.FP64, 1e-12), (lbpc.DF64, 1e-11), (lbpc.FP32, 2e-5)],
                         ids=["fp64", "df64", "fp32"])
def test_split_and_fused_agree(prec, tol):
    """The two kernel organisations compute the same step (they differ only in operation order)."""
    case, rho, T = workloads.mixed_small(TC, RV, RL, nx=67, ny=45)
    a, fa, ga, _ = _gpu(case, rho, T, 50, prec=prec, path=lbpc.PATH_SPLIT)
    b, fb, gb, _ = _gpu(case, rho, T, 50, prec=prec, path=lbpc.PATH_FUSED)
    assert np.max(np.abs(fa - fb)) / np.max(np.abs(fa)) < tol
    assert np.max(np.abs(ga - gb)) / np.max(np.abs(ga)) < tol


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_fp16_deviation_storage(path):
    """Binary16 storage of the deviation from the rest-state equilibrium (FP32 arithmetic) against the
    FP64 oracle. Post-collision populations at the interface deviate from w rho by up to about half
    of w rho, so binary16 (2^-11 relative) limits each step to about 2.7e-4 of a population there; the
    bound below (1e-3 on rho and T after 100 steps) follows from that, and FP32 storage is checked
    beside it against 1e-4."""
    case, rho, T = workloads.droplet_periodic(TC, RV, RL)
    p, s = run_oracle(case, rho, T, 100)
    g16, *_ = _gpu(case, rho, T, 100, prec=lbpc.FP16DEV, path=path)
    e16 = _errors(g16, p, s)
    assert e16["rho"] < 1e-3 and e16["T"] < 1e-3 and e16["ux"] < 2e-2 and e16["uy"] < 2e-2, e16
    g32, *_ = _gpu(case, rho, T, 100, prec=lbpc.FP32, path=path)
    _assert_within(_errors(g32, p, s), 1e-4)


@pytest.mark.parametrize("prec", [lbpc.FP32, lbpc.FP16DEV], ids=["fp32", "fp16"])
def test_persistent_staged_walk_matches(prec):
    """Tile configuration 4 (persistent CTAs, each staging its next tile while it finishes the current
    one) equals configuration 1 bit for bit after 64 steps on grids where it runs persistent (more than 8
    tiles per resident CTA). The grids are a 2048^2 droplet (16384 tiles, about 27 per CTA, edge tiles on the held
    ring) and a 1024 x 2048 pool with walls, a pressure top, a heated strip and the domain-mean buoyancy
    (8192 tiles, so the per-tile partial sums of rho come from CTAs that own several tiles)."""
    for case, rho, T in (workloads.droplet_evaporation(TC, RV, RL, n=2048, radius=400.0, dT_ratio=0.1),
                         workloads.mixed_small(TC, RV, RL, nx=1024, ny=2048)):
        out = []
        for tile in (1, 4):
            sim = lbpc.Simulation(lbpc.params_from_case(case, prec))
            sim.set_fused_tile(tile)
            sim.init(rho, T)
            sim.step(64)
            sim.check()
            out.append(sim.fields())
            sim.close()
        for a, b in zip(out[1], out[0]):
            assert np.array_equal(a, b), case["name"]


@pytest.mark.parametrize("prec", [lbpc.FP32, lbpc.FP16DEV], ids=["fp32", "fp16"])
def test_fused_tile_shapes(prec):
    """Every tile configuration of the fused step (32 x 16 and 32 x 8 with one node per thread, 32 x 16
    and 32 x 32 with two, 32 x 8 in persistent CTAs that stage each next tile early; TMA-staged interior
    tiles) computes the same step; the FP32 result stays
    within 1e-4 of the oracle. A ragged 101 x 75 grid exercises partial tiles and the plain-load path
    (its rows are not 16-byte multiples, so no TMA).

    The configurations with the same nodes per thread run the same code and agree bit for bit. With two
    nodes per thread the compiler fuses some multiplies and adds differently, so the two groups agree to
    binary32 round-off grown over the 60 steps: about 3e-5 relative in FP32. Binary16 storage turns such
    a difference into a rounding of a stored deviation to the other side, 2^-11 of it, so the FP16 groups
    agree to about 1e-4 (the path's own error against the oracle is 2e-2 on u)."""
    between = 5e-5 if prec == lbpc.FP32 else 3e-4
    for case, rho, T in (workloads.droplet_periodic(TC, RV, RL), workloads.mixed_small(TC, RV, RL, nx=101, ny=75)):
        out = []
        for tile in (0, 1, 2, 3, 4):
            sim = lbpc.Simulation(lbpc.params_from_case(case, prec))
            sim.set_fused_tile(tile)
            sim.init(rho, T)
            sim.step(60)
            out.append(sim.fields())
            sim.close()
        for same in ((0, 1), (0, 4), (2, 3)):  # same nodes per thread: the same bits
            for a, b in zip(out[same[1]], out[same[0]]):
                assert np.array_equal(a, b), (case["name"], same)
        for a, b in zip(out[2], out[0]):
            assert np.max(np.abs(a - b)) <= between * np.max(np.abs(b)) + 1e-12, case["name"]
        if prec == lbpc.FP32:
            p, s = run_oracle(case, rho, T, 60)
            for o in out:
                _assert_within(_errors(o, p, s), 1e-4)


def test_sums_async_equals_sums():
    """lbpc_sums_async leaves each step's (mass, heat) in pinned host or device memory without waiting;
    the values equal, bit for bit, lbpc_sums at the same steps of an identical context."""
    import torch

    case, rho, T = workloads.mixed_small(TC, RV, RL)
    a = lbpc.Simulation(lbpc.params_from_case(case))
    b = lbpc.Simulation(lbpc.params_from_case(case))
    a.init(rho, T)
    b.init(rho, T)
    host = torch.zeros((5, 2), dtype=torch.float64).pin_memory()
    dev = torch.zeros(2, dtype=torch.float64, device="cuda")
    want = []
    for k in range(5):
        a.step(2, sync=False)
        a.sums_async(host[k])
        b.step(2)
        want.append(list(b.sums()))
    a.sums_async(dev)
    a.check()
    assert host.tolist() == want
    assert dev.cpu().tolist() == want[-1]
    a.close()
    b.close()


@pytest.mark.parametrize("prec,path", [(lbpc.FP64, lbpc.PATH_SPLIT), (lbpc.FP64, lbpc.PATH_FUSED),
                                       (lbpc.DF64, lbpc.PATH_SPLIT), (lbpc.FP32, lbpc.PATH_FUSED),
                                       (lbpc.FP32, lbpc.PATH_SPLIT), (lbpc.FP16DEV, lbpc.PATH_FUSED)],
                         ids=["fp64-split", "fp64-fused", "df64-split", "fp32-fused", "fp32-split", "fp16-fused"])
def test_no_read_of_unwritten_workspace(monkeypatch, prec, path):
    """Every workspace byte the library does not write itself is NaN (0xFF): the dead population half,
    the scratch planes, phi_prev before the first step, the partial sums. Stepping must give, bit for bit,
    the result of an ordinary workspace. Grids: a ragged 101 x 75 pool with walls, a strip, a pressure top
    and buoyancy, and the closed wettable pool."""
    cases = [workloads.mixed_small(TC, RV, RL, nx=101, ny=75), _closed_wettable_pool()]
    for case, rho, T in cases:
        clean, fc, gc, sc = _gpu(case, rho, T, 7, prec=prec, path=path)
        with monkeypatch.context() as m:
            poison_byte_buffers(m)
            dirty, fd, gd, sd = _gpu(case, rho, T, 7, prec=prec, path=path)
        for a, b in zip(clean, dirty):
            assert np.array_equal(a, b), case["name"]
        assert np.array_equal(fc, fd) and np.array_equal(gc, gd) and sc == sd, case["name"]


def test_poisoning_reaches_the_workspace(monkeypatch):
    """The poisoned workspace of the test above really holds NaN bytes after lbpc_init (in its dead half)."""
    case, rho, T = workloads.mixed_small(TC, RV, RL)
    poison_byte_buffers(monkeypatch)
    sim = lbpc.Simulation(lbpc.params_from_case(case))
    sim.init(rho, T)
    assert int((sim.workspace == 255).sum()) > 0
    sim.close()


@pytest.mark.parametrize("prec", F64, ids=F64_IDS)
@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_buoyancy_referenced_to_the_open_top_fp64(path, prec):
    """Buoyancy 2, F_b = (rho - rho_bc[3]) g under the pressure top, on the ragged mixed grid."""
    case, rho, T = workloads.mixed_small(TC, RV, RL)
    case = dict(case, buoyancy=2)
    gpu, f, _, _ = _gpu(case, rho, T, 150, prec=prec, path=path)
    p, s = _oracle("mixed_small_b2", case, rho, T, 150)
    _assert_within(_errors(gpu, p, s), 1e-10)
    assert np.max(np.abs(f - s.f)) / np.max(np.abs(s.f)) < 1e-10


@pytest.mark.parametrize("path", PATHS, ids=PATH_IDS)
def test_fp32_mass_has_no_systematic_drift(path):
    """Binary32 collisions rebuild the rest population as the zeroth moment minus the others. With the
    plain transform the rounded 1/9 scaled every node's mass by 1 + 7.5e-9 per step: 2.1e-5 after 2000
    steps. Now the drift stays below 5e-6 (measured about 1.8e-6)."""
    case, rho, T = workloads.droplet_periodic(TC, RV, RL, n=64, radius=14.0)
    sim = lbpc.Simulation(lbpc.params_from_case(case, lbpc.FP32))
    sim.set_path(path)
    sim.init(rho, T)
    m0, _ = sim.sums()
    sim.step(2000)
    m1, _ = sim.sums()
    sim.close()
    print(f"FP32 mass drift over 2000 steps ({path}): {(m1 - m0) / m0:.2e}")
    assert abs(m1 - m0) / m0 < 5e-6
