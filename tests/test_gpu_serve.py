"""Continuous-batching service: requests arriving over time are admitted as memory frees up, run
together, and each result is the same as the request run alone (bit for bit: an instance's
arithmetic does not depend on the batch around it)."""

import numpy as np
import pytest

from paper_1709_04400_gb300 import lbpc, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    from paper_1709_04400_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def _stream():
    reqs = serve.poisson_stream(8, rate=200.0, seed=11, side_lo=40, side_hi=96, steps_lo=40, steps_hi=160)
    assert {r.kind for r in reqs} == {"evaporation", "heated_wall"}
    return reqs


def _alone(req, prec=lbpc.FP32):
    srv = serve.Server(prec=prec, hbm_budget_bytes=64 << 20, keep_fields=True)
    (res,) = srv.run([serve.Request(**{**req.__dict__, "arrival": 0.0})])
    srv.close()
    assert res.status == "ok", res.message
    return res.fields


def test_results_same_alone_and_in_the_mix():
    reqs = _stream()
    srv = serve.Server(prec=lbpc.FP32, hbm_budget_bytes=256 << 20, keep_fields=True)
    results = {r.rid: r for r in srv.run(reqs)}
    st = srv.stats()
    srv.close()
    assert st["ok"] == len(reqs) and st["failed"] == 0
    assert st["p50_s"] <= st["p99_s"] and st["aggregate_mlups"] > 0
    for req in reqs:
        res = results[req.rid]
        assert res.steps == req.steps and res.done >= res.admitted >= res.arrival - 1e-9
        for a, e in zip(res.fields, _alone(req)):
            assert np.array_equal(a, e), (req.rid, req.kind)


def test_admission_waits_for_memory():
    """A budget that holds about two requests at a time: every request still completes, later ones
    wait in the queue and join as earlier ones leave (continuous batching)."""
    reqs = serve.poisson_stream(6, rate=1000.0, seed=5, side_lo=64, side_hi=64, steps_lo=50, steps_hi=50)
    case, _, _ = serve.make_case(reqs[0], *_eos())
    per = lbpc.Batch.instance_bytes(lbpc.params_from_case(case, lbpc.FP32))
    srv = serve.Server(prec=lbpc.FP32, hbm_budget_bytes=2 * per + (3 << 20), max_instances=16)
    results = srv.run(reqs)
    srv.close()
    assert all(r.status == "ok" for r in results)
    waited = [r for r in results if r.admitted - r.arrival > 1e-4]
    assert len(waited) >= 2


def _eos():
    p0 = lbpc.Params(nx=8, ny=8)
    Tc, _ = lbpc.eos_critical(p0)
    rv, rl, _ = lbpc.coexistence(p0, 0.86 * Tc)
    return Tc, rv, rl


def test_failed_request_retired_while_others_complete(monkeypatch):
    """A request whose initial state holds a density beyond the EOS pole fails after the first chunk
    with the steps it ran; the requests around it complete and equal their runs alone."""
    reqs = _stream()[:4]
    bad = reqs[1].rid
    real = serve.make_case

    def planted(req, *a):
        case, rho, T = real(req, *a)
        if req.rid == bad:
            rho = rho.copy()
            rho[3, 5] = 11.0
        return case, rho, T

    monkeypatch.setattr(serve, "make_case", planted)
    srv = serve.Server(prec=lbpc.FP32, hbm_budget_bytes=256 << 20, max_chunk=16, keep_fields=True)
    results = {r.rid: r for r in srv.run([serve.Request(**{**r.__dict__, "arrival": 0.0}) for r in reqs])}
    st = srv.stats()
    srv.close()
    assert results[bad].status == "failed" and results[bad].message == "non-physical state"
    assert 0 < results[bad].steps <= 16
    assert st["failed"] == 1 and st["ok"] == len(reqs) - 1
    monkeypatch.setattr(serve, "make_case", real)
    for req in reqs:
        if req.rid != bad:
            res = results[req.rid]
            assert res.status == "ok" and res.steps == req.steps
            for a, e in zip(res.fields, _alone(req)):
                assert np.array_equal(a, e), req.rid
