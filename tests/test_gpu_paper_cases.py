"""The paper's droplet-evaporation case (Sec. IV A, Figs. 1-2) on the GPU with the three thermal models.

Fig. 2 states that (D/D0)^2 falls linearly in time for the compromised and improved models (the D^2
law), with visible differences between the two. It also states that the Gong-Cheng model evaporates
much faster and does not follow the law. Sec. IV A adds that with a constant lambda the Gong-Cheng
evaporation is the fastest. The figure data are not in the paper's text, so these tests check the
paper's qualitative statements.

The Gong-Cheng model is a BGK step with tau_g = lambda/(rho c_s^2 c_V) + 1/2 (Eq. 12). At the
paper's lambda = 2/3 this gives tau_g = 0.56 in the liquid, and the droplet centre diverges a few
hundred steps in. The oracle diverges at the same step and node. So the speed comparison runs at
lambda = 1 (tau_g = 0.59 in the liquid), where all three models are stable. At the divergence step
a single node fails, so the reported node is unique."""

import numpy as np
import pytest

from paper_1709_04400_gb300 import lbpc, workloads

from .helpers import RL, RV, TC, contact_angle, departed_bubble, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    from paper_1709_04400_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _d2_history(model, lam=2.0 / 3.0, steps=40000, every=2000):
    case, rho, T = workloads.paper_d2_law(TC, RV, RL, model=model, lam=lam)
    sim = lbpc.Simulation(lbpc.params_from_case(case, lbpc.FP64))
    sim.init(rho, T)
    a0 = workloads.droplet_area(sim.fields()[0])
    ts, d2 = [0], [1.0]
    for k in range(steps // every):
        sim.step(every)
        ts.append((k + 1) * every)
        d2.append(workloads.droplet_area(sim.fields()[0]) / a0)
    sim.close()
    return np.array(ts), np.array(d2)


def _linear_fit(t, y):
    c = np.polyfit(t, y, 1)
    return c[0], 1 - ((y - np.polyval(c, t)) ** 2).sum() / ((y - y.mean()) ** 2).sum()


def test_d2_law_improved_and_compromised():
    """Paper set-up (lambda = 2/3): linear (D/D0)^2 after the start-up transient (t >= 10^4), R^2 > 0.99,
    and a visible difference between the two models."""
    end = {}
    for m in ("improved", "compromised"):
        t, d2 = _d2_history(m)
        sel = t >= 10000
        slope, r2 = _linear_fit(t[sel], d2[sel])
        print(f"{m}: (D/D0)^2 at t = {t[-1]}: {d2[-1]:.4f}, slope {slope:.3e} per step, R^2 {r2:.5f}")
        assert slope < 0 and r2 > 0.99, m
        end[m] = d2[-1]
    assert abs(end["improved"] - end["compromised"]) > 0.005


def test_gong_cheng_evaporates_fastest_at_constant_lambda():
    """Constant lambda = 1: the Gong-Cheng droplet loses several times the area the improved model's loses."""
    _, d_imp = _d2_history("improved", lam=1.0)
    _, d_cmp = _d2_history("compromised", lam=1.0)
    _, d_gc = _d2_history("gong_cheng", lam=1.0)
    print(f"lambda = 1, (D/D0)^2 at t = 40000: improved {d_imp[-1]:.4f}, compromised {d_cmp[-1]:.4f}, "
          f"Gong-Cheng {d_gc[-1]:.4f}")
    assert (1 - d_gc[-1]) > 3 * (1 - d_imp[-1]) and (1 - d_gc[-1]) > 3 * (1 - d_cmp[-1])


def test_gong_cheng_divergence_matches_oracle():
    """At the paper's lambda = 2/3 the Gong-Cheng step diverges at the droplet centre; the GPU reports the
    oracle's step and node."""
    from oracle import model

    case, rho, T = workloads.paper_d2_law(TC, RV, RL, model="gong_cheng")
    p = oracle_params(case)
    s = model.init_state(p, rho, T)
    with pytest.raises(model.OracleNonPhysical) as eo:
        for _ in range(1000):
            s = model.step(p, s)
    sim = lbpc.Simulation(lbpc.params_from_case(case, lbpc.FP64))
    sim.init(rho, T)
    with pytest.raises(lbpc.LbpcError) as eg:
        sim.step(1000)
    sim.close()
    assert eg.value.status == lbpc.LBPC_ENONPHYS
    o = eo.value
    assert f"step {o.step}, node (x={o.x}, y={o.y})" in str(eg.value), (str(eo.value), str(eg.value))


def test_heated_strip_nucleates_vapour():
    """Sec. IV B, qualitatively: liquid over a wall at T_sat with a hotter strip (here the closed pool of
    the heated-wall workload, strip T_s + 0.3 T_c). Vapour must form over the strip, on the wall, and
    nowhere else along the wall, and the FP32 step must show the same vapour region as FP64. Neither
    the contact-angle scheme nor the top boundary is named in the paper, so the departure diameter of
    Fig. 7 is not compared."""
    from scipy import ndimage

    case, rho, T = workloads.heated_wall(TC, RV, RL, top="wall")
    x0, x1, _ = case["strip"]
    mid = 0.5 * (RV + RL)
    areas = {}
    for prec in (lbpc.FP64, lbpc.FP32):
        sim = lbpc.Simulation(lbpc.params_from_case(case, prec))
        sim.init(rho, T)
        sim.step(1000)
        r = sim.fields()[0]
        sim.close()
        ny = r.shape[0]
        lab, n = ndimage.label(r[: ny // 2 - 20] < mid)  # vapour below the free surface
        assert n >= 1, prec
        sizes = ndimage.sum(np.ones_like(lab), lab, index=range(1, n + 1))
        big = 1 + int(np.argmax(sizes))
        ys, xs = np.nonzero(lab == big)
        assert ys.min() == 0, "the vapour region sits on the wall"
        assert x0 - 15 <= xs.min() and xs.max() < x1 + 15, (xs.min(), xs.max(), x0, x1)
        assert r[1:6, : x0 - 40].min() > 0.9 * RL and r[1:6, x1 + 40:].min() > 0.9 * RL, "far wall stays liquid"
        areas[prec] = sizes.max()
    assert abs(areas[lbpc.FP32] - areas[lbpc.FP64]) <= 0.05 * areas[lbpc.FP64], areas


def test_departure_diameter_follows_inverse_root_of_gravity():
    """Fig. 7: the departure diameter falls as g^(-1/2), D_d = 0.209 g^(-1/2) in the paper. The pool of
    workloads.bubble_departure, with the paper's 45-degree contact angle (G_wall = -0.17 under this
    build's adsorption force, calibrated on a sessile droplet), is run at g from 4e-5 to 2e-4 (a factor
    of 5); measured D_d = 0.234 g^(-1/2), fitted 0.212 g^-0.511. D_d = 2 sqrt(A/pi) of the
    region that detaches, at the first check (every 20 steps) after it leaves the wall. The fitted
    exponent must lie within 0.1 of -1/2 and the prefactor within 25 % of 0.209 (the contact-angle
    scheme and the top boundary of the paper's set-up are not stated, so the prefactor can differ)."""
    gs = [4e-5, 6e-5, 1e-4, 1.4e-4, 2e-4]
    dd = []
    for g in gs:
        case, rho, T = workloads.bubble_departure(TC, RV, RL, g=g, G_wall=-0.17)
        sim = lbpc.Simulation(lbpc.params_from_case(case, lbpc.FP64))
        sim.init(rho, T)
        area = 0
        while not area and sim.step_count < 60000:
            sim.step(20)
            area = departed_bubble(sim.fields()[0], case["surface"])
        sim.close()
        assert area, g
        dd.append(2.0 * np.sqrt(area / np.pi))
    slope, lnc = np.polyfit(np.log(gs), np.log(dd), 1)
    c_half = float(np.mean(np.array(dd) * np.sqrt(gs)))  # prefactor with the exponent fixed at -1/2
    print(f"departure diameters {dict(zip(gs, np.round(dd, 2)))}: fit D_d = {np.exp(lnc):.3f} g^{slope:.3f}; "
          f"with exponent -1/2, D_d = {c_half:.3f} g^-0.5 (paper 0.209)")
    assert abs(slope + 0.5) <= 0.1
    assert abs(c_half / 0.209 - 1.0) <= 0.25


def _departure(model, g):
    case, rho, T = workloads.bubble_departure(TC, RV, RL, g=g)
    sim = lbpc.Simulation(lbpc.params_from_case(dict(case, model=model), lbpc.FP64))
    sim.init(rho, T)
    area = 0
    while not area and sim.step_count < 30000:
        sim.step(20)
        area = departed_bubble(sim.fields()[0], case["surface"])
    step = sim.step_count
    sim.close()
    return (step, 2.0 * np.sqrt(area / np.pi)) if area else (None, 0.0)


def test_models_differ_in_bubble_departure():
    """Figs. 5-6, qualitatively: the Gong-Cheng model deviates strongly from the other two (here its
    bubble departs at less than 0.6 of the improved model's time with a diameter 1.2 times larger or
    more; measured 4360 against 9440 steps, 30.9 against 23.1 nodes at g = 1e-4), and the compromised
    model differs visibly from the improved one (its departure comes at least 5 % later; measured 10540)."""
    g = 1e-4
    imp, com, gc = (_departure(m, g) for m in ("improved", "compromised", "gong_cheng"))
    print(f"departure at g = {g}: improved {imp}, compromised {com}, Gong-Cheng {gc} (step, D_d)")
    assert imp[0] and com[0] and gc[0]
    assert gc[0] < 0.6 * imp[0] and gc[1] > 1.2 * imp[1]
    assert com[0] > 1.05 * imp[0]


def _relaxed_droplet_on_surface(G_wall):
    """The droplet of workloads.droplet_on_surface after the paper's 20 000 isothermal steps."""
    case, rho, T = workloads.droplet_on_surface(TC, RV, RL, G_wall=G_wall)
    sim = lbpc.Simulation(lbpc.params_from_case(case, lbpc.FP64))
    sim.init(rho, T)
    sim.step(20000)
    out = sim.fields()
    sim.close()
    return out


def test_droplet_on_surface_evaporation_by_model():
    """Sec. IV A, droplet on a solid surface (Fig. 3). First, 20 000 isothermal steps: the neutral wall
    gives 90 degrees and G_wall = 0.08 gives the paper's 108 degrees (calibrated here). Then the wall is
    heated to 0.875 T_c and the droplet evaporates for 40 000 steps under each model. With
    lambda = rho c_V chi (chi = 0.08) the Gong-Cheng model evaporates slowest; with a constant lambda
    (here 1) it evaporates fastest, as the paper reports. Rates are the slopes of the droplet area over
    steps 4000-40000. Measured: variable lambda, Gong-Cheng 0.67 of the improved model's rate; constant
    lambda, 1.84 of it and 1.30 of the compromised model's."""
    neutral = _relaxed_droplet_on_surface(0.0)
    assert abs(contact_angle(neutral[0]) - 90.0) <= 2.0
    rho0, ux0, uy0, T0 = _relaxed_droplet_on_surface(0.08)
    theta = contact_angle(rho0)
    mid = 0.5 * (RL + RV)
    rates = {}
    for lm in ("rho_cv_chi", "const"):
        for model in ("improved", "compromised", "gong_cheng"):
            case, _, _ = workloads.droplet_on_surface(TC, RV, RL, G_wall=0.08, wall_T_ratio=0.875, lambda_mode=lm,
                                                      model=model)
            sim = lbpc.Simulation(lbpc.params_from_case(case, lbpc.FP64))
            sim.init(rho0, T0, ux0, uy0)
            sim.step(4000)
            t, area = [], []
            for k in range(4000, 40001, 2000):
                if k > 4000:
                    sim.step(2000)
                t.append(k)
                area.append(float((sim.fields()[0] > mid).sum()))
            sim.close()
            rates[(lm, model)] = -np.polyfit(t, area, 1)[0]
    print(f"contact angle {theta:.1f} deg; evaporation rates (area per step): "
          + ", ".join(f"{k[0]}/{k[1]} {v:.2e}" for k, v in rates.items()))
    assert abs(theta - 108.0) <= 3.0
    assert all(v > 0 for v in rates.values())
    v = lambda lm, m: rates[(lm, m)]  # noqa: E731
    assert v("rho_cv_chi", "gong_cheng") < 0.8 * v("rho_cv_chi", "improved")
    assert v("rho_cv_chi", "gong_cheng") < v("rho_cv_chi", "compromised")
    assert v("const", "gong_cheng") > 1.3 * v("const", "improved")
    assert v("const", "gong_cheng") > 1.1 * v("const", "compromised")


def test_bench_workload_follows_the_d2_law():
    """The bench workload itself (256^2, R = 40, superheat dT in {0.05, 0.1, 0.2} T_c held on the outer
    ring). Heat reaches the droplet by diffusion through about 88 nodes of vapour, with
    chi_v = lambda/(rho_v c_V) = 0.35: a start-up time of order L^2/chi_v = 2.2e4 steps, during which the
    droplet first grows slightly. After it, over steps 30 000-60 000, (D/D0)^2 falls linearly
    (R^2 > 0.98; measured 0.990, 0.998, 0.999), faster the larger the superheat (slopes -1.7e-7,
    -6.4e-7, -1.39e-6 per step)."""
    slopes = {}
    for dT in (0.05, 0.1, 0.2):
        case, rho, T = workloads.droplet_evaporation(TC, RV, RL, n=256, radius=40.0, dT_ratio=dT)
        sim = lbpc.Simulation(lbpc.params_from_case(case, lbpc.FP64))
        sim.init(rho, T)
        a0 = workloads.droplet_area(sim.fields()[0])
        ts, d2 = [], []
        for k in range(1, 61):
            sim.step(1000)
            ts.append(1000 * k)
            d2.append(workloads.droplet_area(sim.fields()[0]) / a0)
        sim.close()
        t, y = np.array(ts), np.array(d2)
        sel = t >= 30000
        slope, r2 = _linear_fit(t[sel], y[sel])
        print(f"dT = {dT} T_c: (D/D0)^2 at 60000 steps {y[-1]:.4f}, slope {slope:.3e} per step, R^2 {r2:.5f}; "
              f"every 6000 steps {np.round(y[5::6], 4).tolist()}")
        slopes[dT] = (slope, r2)
    for dT, (slope, r2) in slopes.items():
        assert slope < 0 and r2 > 0.98, (dT, slope, r2)
    assert slopes[0.2][0] < slopes[0.1][0] < slopes[0.05][0]


def test_heated_wall_with_open_top_runs_30000_steps():
    """The heated-wall nucleation workload as specified: 300 x 400 pool, heated strip, wall at y = 0, the
    top held at the vapour density and T_s, g = 3e-5, FP32, 30 000 steps. With the buoyancy referenced to the top's density
    (buoyancy 2, the workload's default under this top) the run stays physical, keeps its mass within
    1e-3 and holds a vapour region on the wall over the strip. With the domain mean as the reference it
    leaves the EOS range after about 1850 steps (both the oracle and the GPU)."""
    from scipy import ndimage

    case, rho, T = workloads.heated_wall(TC, RV, RL)
    assert case["buoyancy"] == 2
    sim = lbpc.Simulation(lbpc.params_from_case(case, lbpc.FP32))
    sim.init(rho, T)
    m0 = float(rho.sum())
    sim.step(30000)
    sim.check()
    r = sim.fields()[0]
    sim.close()
    assert abs(r.sum() - m0) / m0 < 1e-3
    lab, n = ndimage.label(r[:180] < 0.5 * (RL + RV))
    x0, x1, _ = case["strip"]
    on_wall = [j for j in range(1, n + 1) if np.nonzero(lab == j)[0].min() == 0]
    assert on_wall
    xs = np.nonzero(np.isin(lab, on_wall))[1]
    assert x0 - 15 <= xs.min() and xs.max() < x1 + 15
