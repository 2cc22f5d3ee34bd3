"""Batched step (lbpc_batch_*): many instances of uneven size in one persistent launch per step.

An instance's result must not depend on what else is in the batch: each one is checked bit for bit
against the same instance in a batch of its own, and to round-off against the single-instance entry
point (lbpc_create / lbpc_step, fused path). The oracle bounds the FP32 batch to 1e-4 and the FP64
batch to 1e-10 as elsewhere."""

import numpy as np
import pytest

from paper_1709_04400_gb300 import inputs, lbpc, workloads

from .helpers import RL, RV, TC, TS, max_rel, norm_rel, poison_byte_buffers, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    from paper_1709_04400_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _cases():
    """Uneven sizes and every boundary class."""
    out = []
    out.append(workloads.mixed_small(TC, RV, RL, nx=37, ny=29))
    out.append(workloads.droplet_periodic(TC, RV, RL, n=64, radius=14.0))
    out.append(workloads.droplet_evaporation(TC, RV, RL, n=96, radius=20.0, dT_ratio=0.2))
    out.append(workloads.heated_wall(TC, RV, RL, nx=70, ny=90, strip_width=8))
    out.append(workloads.mixed_small(TC, RV, RL, nx=33, ny=17))
    return out


def _alone(case, rho, T, steps, prec):
    sim = lbpc.Simulation(lbpc.params_from_case(case, prec))
    sim.set_path(lbpc.PATH_FUSED)
    sim.init(rho, T)
    sim.step(steps)
    out = sim.fields()
    sim.close()
    return out


def _solo(case, rho, T, steps, prec, config=None):
    """The instance in a batch of its own (default configuration, or config = (variant, ctas per SM))."""
    b = lbpc.Batch(prec, _arena_for([(case, rho, T)], prec))
    if config is not None:
        b.set_config(*config)
    i = b.add(lbpc.params_from_case(case, prec), rho, T)
    b.step(steps)
    out = b.fields(i)
    b.close()
    return out


def _arena_for(cases, prec, extra=64 << 20):
    return sum(lbpc.Batch.instance_bytes(lbpc.params_from_case(c, prec)) for c, _, _ in cases) + extra


TOL_VS_SINGLE = {lbpc.FP32: 1e-5, lbpc.FP16DEV: 2e-3, lbpc.FP64: 1e-13}


@pytest.mark.parametrize("prec", [lbpc.FP32, lbpc.FP16DEV, lbpc.FP64], ids=["fp32", "fp16", "fp64"])
def test_batch_equals_alone(prec):
    """Each instance of a mixed batch equals, bit for bit, the same instance in a batch of its own; and
    it matches the single-instance entry point (a different tile shape of the same arithmetic, where
    the compiler may contract multiply-adds differently) to a round-off tolerance."""
    cases = _cases()
    steps = 40  # two graph chunks of 16 plus 8 direct launches
    b = lbpc.Batch(prec, _arena_for(cases, prec))
    ids = [b.add(lbpc.params_from_case(c, prec), r, t) for c, r, t in cases]
    b.step(steps)
    b.check()
    for i, (c, r, t) in zip(ids, cases):
        got = b.fields(i)
        assert b.step_count(i) == steps
        solo = lbpc.Batch(prec, _arena_for([(c, r, t)], prec))
        j = solo.add(lbpc.params_from_case(c, prec), r, t)
        solo.step(steps)
        for a, e in zip(got, solo.fields(j)):
            assert np.array_equal(a, e), c["name"]
        solo.close()
        ref = _alone(c, r, t, steps, prec)
        tol = TOL_VS_SINGLE[prec]
        assert max_rel(got[0], ref[0]) < tol and max_rel(got[3], ref[3]) < tol, c["name"]
        assert norm_rel(got[1], ref[1]) < 100 * tol and norm_rel(got[2], ref[2]) < 100 * tol, c["name"]
    b.close()


def test_batch_fp32_and_fp64_against_oracle():
    case, rho, T = workloads.mixed_small(TC, RV, RL, nx=37, ny=29)
    p, s = run_oracle(case, rho, T, 60)
    from oracle import model

    r_o, ux_o, uy_o, T_o = model.fields(p, s)
    for prec, tol in ((lbpc.FP32, 1e-4), (lbpc.FP64, 1e-10)):
        b = lbpc.Batch(prec, _arena_for([(case, rho, T)], prec))
        i = b.add(lbpc.params_from_case(case, prec), rho, T)
        b.step(60)
        r, ux, uy, TT = b.fields(i)
        b.close()
        assert max_rel(r, r_o) < tol and max_rel(TT, T_o) < tol
        assert norm_rel(ux, ux_o) < tol and norm_rel(uy, uy_o) < tol


def test_instances_join_and_leave():
    """B joins after A has run 10 steps; A leaves after 20; B's result equals B run alone."""
    prec = lbpc.FP32
    (ca, ra, ta), (cb, rb, tb) = _cases()[1], _cases()[2]
    b = lbpc.Batch(prec, _arena_for([(ca, ra, ta), (cb, rb, tb)], prec))
    ia = b.add(lbpc.params_from_case(ca, prec), ra, ta)
    b.step(10)
    ib = b.add(lbpc.params_from_case(cb, prec), rb, tb)
    b.step(10)
    got_a = b.fields(ia)
    b.remove(ia)
    b.step(22)
    got_b = b.fields(ib)
    b.close()
    for a, e in zip(got_a, _solo(ca, ra, ta, 20, prec)):
        assert np.array_equal(a, e)
    for a, e in zip(got_b, _solo(cb, rb, tb, 32, prec)):
        assert np.array_equal(a, e)


def test_autotune_keeps_results():
    prec = lbpc.FP32
    cases = _cases()[:3]
    b = lbpc.Batch(prec, _arena_for(cases, prec))
    ids = [b.add(lbpc.params_from_case(c, prec), r, t) for c, r, t in cases]
    best = b.autotune(steps_per_candidate=2)
    n = b.step_count(ids[0])
    assert n > 0 and best["ms_per_step"] > 0
    b.step(5)
    for i, (c, r, t) in zip(ids, cases):
        got, ref = b.fields(i), _solo(c, r, t, n + 5, prec)
        assert max_rel(got[0], ref[0]) < 1e-5 and max_rel(got[3], ref[3]) < 1e-5
    b.close()


def test_arena_full_and_slot_reuse():
    prec = lbpc.FP32
    case, rho, T = workloads.droplet_periodic(TC, RV, RL, n=64, radius=14.0)
    per = lbpc.Batch.instance_bytes(lbpc.params_from_case(case, prec))
    b = lbpc.Batch(prec, 2 * per + (64 << 10), max_instances=8)  # room for the descriptors, not a third instance
    i1 = b.add(lbpc.params_from_case(case, prec), rho, T)
    i2 = b.add(lbpc.params_from_case(case, prec), rho, T)
    with pytest.raises(lbpc.LbpcError) as e:
        b.add(lbpc.params_from_case(case, prec), rho, T)
    assert e.value.status == lbpc.LBPC_ENOMEM
    b.remove(i1)
    i3 = b.add(lbpc.params_from_case(case, prec), rho, T)
    assert i3 == i1
    b.step(3)
    assert b.step_count(i3) == 3 and b.step_count(i2) == 3
    b.close()


def test_failed_instance_named_and_others_unaffected():
    """One instance starts with a density beyond the EOS pole (1/b = 10.5). The check names that instance
    and the first bad node. Once it is removed, the check passes again, and the other instances
    equal, bit for bit, their runs in batches of their own."""
    prec = lbpc.FP32
    cases = _cases()[:3]
    bad_case, bad_rho, bad_T = workloads.droplet_periodic(TC, RV, RL, n=32, radius=8.0)
    bad_rho = bad_rho.copy()
    bad_rho[7, 11] = 11.0
    b = lbpc.Batch(prec, _arena_for(cases + [(bad_case, bad_rho, bad_T)], prec))
    ids = [b.add(lbpc.params_from_case(c, prec), r, t) for c, r, t in cases[:2]]
    ib = b.add(lbpc.params_from_case(bad_case, prec), bad_rho, bad_T)
    ids.append(b.add(lbpc.params_from_case(cases[2][0], prec), cases[2][1], cases[2][2]))
    b.step(5)
    with pytest.raises(lbpc.LbpcError) as e:
        b.check()
    assert e.value.status == lbpc.LBPC_ENONPHYS and e.value.instance == ib
    assert f"instance {ib}: non-physical state at step 0, node (x=11, y=7)" in str(e.value)
    b.remove(ib)
    b.check()
    b.step(7)
    for i, (c, r, t) in zip(ids, cases):
        assert b.step_count(i) == 12
        for a, ex in zip(b.fields(i), _solo(c, r, t, 12, prec)):
            assert np.array_equal(a, ex), c["name"]
    b.close()


@pytest.mark.parametrize("prec", [lbpc.FP32, lbpc.FP16DEV, lbpc.FP64], ids=["fp32", "fp16", "fp64"])
def test_no_read_of_unwritten_arena(monkeypatch, prec):
    """The arena filled with 0xFF bytes (NaN in every storage type) before the batch is created: every
    byte the library does not write itself stays NaN. The batch of mixed instances must step to the same
    bits as in an ordinary arena, with the default and a tuned configuration."""
    cases = _cases()

    def run(tune):
        b = lbpc.Batch(prec, _arena_for(cases, prec))
        ids = [b.add(lbpc.params_from_case(c, prec), r, t) for c, r, t in cases]
        if tune:
            b.set_config(3, 8)
        b.step(20)
        b.check()
        out = [b.fields(i) for i in ids]
        b.close()
        return out

    for tune in (False, True):
        clean = run(tune)
        with monkeypatch.context() as m:
            poison_byte_buffers(m)
            dirty = run(tune)
        for fc, fd in zip(clean, dirty):
            for a, b in zip(fc, fd):
                assert np.array_equal(a, b), tune


@pytest.mark.parametrize("prec", [lbpc.FP32, lbpc.FP16DEV, lbpc.FP64], ids=["fp32", "fp16", "fp64"])
def test_per_tile_launches(prec):
    """Per-tile launches (0 CTAs per SM: one CTA per tile, the instances in the kernel parameters). The
    steps are taken as 17 + 16 + 3, so graphs of 16 steps replay at both step parities and single steps
    run between them. Each instance of the mixed batch equals, bit for bit, the same instance in a batch
    of its own in this configuration stepped 36 times at once. It matches the work-list kernel of the
    same tile shape to round-off."""
    cases = _cases()
    b = lbpc.Batch(prec, _arena_for(cases, prec))
    b.set_config(0, 0)
    ids = [b.add(lbpc.params_from_case(c, prec), r, t) for c, r, t in cases]
    for n in (17, 16, 3):
        b.step(n)
    b.check()
    tol = TOL_VS_SINGLE[prec]
    for i, (c, r, t) in zip(ids, cases):
        got = b.fields(i)
        assert b.step_count(i) == 36
        for a, e in zip(got, _solo(c, r, t, 36, prec, config=(0, 0))):
            assert np.array_equal(a, e), c["name"]
        ref = _solo(c, r, t, 36, prec, config=(0, 8))
        assert max_rel(got[0], ref[0]) < tol and max_rel(got[3], ref[3]) < tol, c["name"]
        assert norm_rel(got[1], ref[1]) < 100 * tol and norm_rel(got[2], ref[2]) < 100 * tol, c["name"]
    b.close()


def test_per_tile_launches_many_instances_join_and_leave():
    """More instances than one per-tile launch holds (so a step takes several launches), instances that
    join and leave between steps, and every remaining instance equal, bit for bit, to its run alone."""
    prec = lbpc.FP32
    cap = lbpc.Batch.per_tile_capacity(prec)
    small = [workloads.droplet_periodic(TC, RV, RL, n=24 + 2 * (k % 5), radius=6.0) for k in range(cap + 6)]
    b = lbpc.Batch(prec, _arena_for(small, prec), max_instances=len(small) + 2)
    b.set_config(0, 0)
    ids = [b.add(lbpc.params_from_case(c, prec), r, t) for c, r, t in small[:-3]]
    b.step(19)
    late = [b.add(lbpc.params_from_case(c, prec), r, t) for c, r, t in small[-3:]]
    b.remove(ids[1])
    b.step(20)
    b.check()
    for k, i in enumerate(ids):
        if k == 1:
            continue
        c, r, t = small[k]
        for a, e in zip(b.fields(i), _solo(c, r, t, 39, prec, config=(0, 0))):
            assert np.array_equal(a, e), k
    for k, i in enumerate(late):
        c, r, t = small[len(small) - 3 + k]
        for a, e in zip(b.fields(i), _solo(c, r, t, 20, prec, config=(0, 0))):
            assert np.array_equal(a, e), k
    b.close()


@pytest.mark.parametrize("config", [(0, 0), (0, 8)], ids=["per-tile", "work-list"])
@pytest.mark.parametrize("prec,tol", [(lbpc.FP64, 1e-10), (lbpc.FP32, 1e-4)], ids=["fp64", "fp32"])
def test_tiny_and_narrow_instances_against_oracle(config, prec, tol):
    """Instances smaller than one tile or narrower than the ring (2 x 3, 3 x 64, 200 x 3, a 6 x 6 periodic
    droplet), where every tile is an edge tile, indices wrap several times and partial tiles hold a few
    nodes, side by side in one batch in both launch forms: each against the oracle after 20 steps. The
    velocity error is relative to max(max |u|, 1e-3): in the 2-wide domain u_x stays near 1e-6 by
    symmetry, below the binary32 rounding of the momentum (about 4e-9 at these densities) times 1e3."""
    def vapour(nx, ny):  # every boundary class on a grid too small for a liquid region: vapour near saturation
        case, _, _ = workloads.mixed_small(TC, RV, RL, nx=nx, ny=ny)
        return case, RV * (1.0 + 0.01 * (np.arange(nx * ny) % 7).reshape(ny, nx)), np.full((ny, nx), TS)

    cases = [vapour(2, 3), workloads.mixed_small(TC, RV, RL, nx=3, ny=64), vapour(200, 3),
             workloads.droplet_periodic(TC, RV, RL, n=6, radius=2.0)]
    steps = 20
    b = lbpc.Batch(prec, _arena_for(cases, prec))
    b.set_config(*config)
    ids = [b.add(lbpc.params_from_case(c, prec), r, t) for c, r, t in cases]
    b.step(steps)
    b.check()
    from oracle import model

    for i, (c, r, t) in zip(ids, cases):
        p, s = run_oracle(c, r, t, steps)
        ref = model.fields(p, s)
        got = b.fields(i)
        u_scale = max(float(np.max(np.abs(ref[1]))), float(np.max(np.abs(ref[2]))), 1e-3)
        err = dict(rho=max_rel(got[0], ref[0]), T=max_rel(got[3], ref[3]),
                   u=max(float(np.max(np.abs(got[1] - ref[1]))), float(np.max(np.abs(got[2] - ref[2])))) / u_scale)
        assert all(v <= tol for v in err.values()), (c["name"], err)
    b.close()
