"""Host logic of the continuous-batching service (serve.Server), on the CPU with a fake batch.

The fake stands in for lbpc.Batch: it accounts bytes against a budget, counts steps per instance and
reports scripted non-physical failures. It computes no physics. The scheduler must do the following.
- Admit requests in arrival order, each once it has arrived and the budget has room.
- Keep a request that can never fit out of the batch and report it failed.
- Advance in chunks no longer than the shortest remaining request (capped).
- Retire a failed instance while the others carry on.
- Return every request exactly once, with the steps it asked for."""

import itertools

import numpy as np
import pytest

from paper_1709_04400_gb300 import lbpc, serve


class FakeClock:
    """Deterministic clock: every call advances by dt seconds."""

    def __init__(self, dt=1e-3):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeBatch:
    instances = []  # every FakeBatch created, for inspection

    def __init__(self, prec, arena_bytes, max_instances=4096, device=None, high_priority=False):
        self.budget = int(arena_bytes)
        self.used = {}
        self.steps = {}
        self.fail_at = {}  # instance id -> step count at which it turns non-physical
        self.ids = itertools.count()
        self.log = []  # (event, id, value)
        self.max_active = 0
        FakeBatch.instances.append(self)

    @staticmethod
    def instance_bytes(p):
        return p.nx * p.ny * 100

    def free_bytes(self):
        return self.budget - sum(self.used.values())

    def add(self, p, rho, T):
        need = FakeBatch.instance_bytes(p)
        if need > self.free_bytes():
            raise lbpc.LbpcError(lbpc.LBPC_ENOMEM, "fake arena full")
        i = next(self.ids)
        self.used[i] = need
        self.steps[i] = 0
        self.max_active = max(self.max_active, len(self.used))
        self.log.append(("add", i, p.nx))
        return i

    def remove(self, i):
        self.log.append(("remove", i, self.steps[i]))
        del self.used[i]

    def step(self, n):
        self.log.append(("step", -1, n))
        for i in self.used:
            self.steps[i] += n

    def check(self):
        for i in sorted(self.used):
            if i in self.fail_at and self.steps[i] >= self.fail_at[i]:
                e = lbpc.LbpcError(lbpc.LBPC_ENONPHYS, f"fake instance {i} non-physical")
                e.instance = i
                raise e

    def fields(self, i):
        return None

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    FakeBatch.instances = []
    monkeypatch.setattr(lbpc, "Batch", FakeBatch)
    return FakeBatch


def _req(rid, side, steps, arrival, kind="evaporation"):
    return serve.Request(rid, kind, side, steps, side * 0.2 if kind == "evaporation" else 4, 0.1, arrival)


def test_all_requests_served_once_with_their_steps(fake):
    reqs = serve.poisson_stream(40, rate=200.0, seed=7, side_lo=16, side_hi=48, steps_lo=10, steps_hi=200)
    srv = serve.Server(prec=lbpc.FP32, hbm_budget_bytes=1 << 30, max_chunk=64, clock=FakeClock())
    res = srv.run(reqs)
    assert sorted(r.rid for r in res) == list(range(40))
    by = {r.rid: r for r in reqs}
    for r in res:
        assert r.status == "ok" and r.steps == by[r.rid].steps
        assert r.admitted >= by[r.rid].arrival - 1e-9  # never admitted before it arrived
        assert r.done >= r.admitted
    b = fake.instances[0]
    chunks = [v for e, _, v in b.log if e == "step"]
    assert max(chunks) <= 64 and min(chunks) >= 1
    st = srv.stats()
    assert st["ok"] == 40 and st["failed"] == 0 and st["p99_s"] >= st["p50_s"] > 0


def test_budget_gates_admission_in_arrival_order(fake):
    per = 32 * 32 * 100
    # room for two 32^2 requests at a time; five arrive at once
    reqs = [_req(k, 32, 50 + 10 * k, 0.0) for k in range(5)]
    srv = serve.Server(prec=lbpc.FP32, hbm_budget_bytes=2 * per + (1 << 20), max_chunk=1000, clock=FakeClock())
    srv.run(reqs)
    b = fake.instances[0]
    adds = [i for e, i, _ in b.log if e == "add"]
    assert b.max_active <= 2
    assert adds == sorted(adds)  # first in, first admitted
    # every admission after the first two waits for a removal
    events = [e for e, _, _ in b.log if e in ("add", "remove")]
    assert events[:2] == ["add", "add"] and events[2] == "remove"


def test_request_that_can_never_fit_fails_alone(fake):
    small, big = _req(0, 16, 40, 0.0), _req(1, 512, 40, 0.0)
    srv = serve.Server(prec=lbpc.FP32, hbm_budget_bytes=(1 << 20) + 64 * 64 * 100, clock=FakeClock())
    res = {r.rid: r for r in srv.run([big, small])}
    assert res[1].status == "failed" and "needs" in res[1].message
    assert res[0].status == "ok" and res[0].steps == 40


def test_failed_instance_is_retired_and_others_continue(fake):
    reqs = [_req(k, 24, 300, 0.0) for k in range(4)]
    orig_init = FakeBatch.__init__

    def init(self, *a, **kw):
        orig_init(self, *a, **kw)
        self.fail_at = {1: 100}  # the second admitted instance turns non-physical at step 100

    fake.__init__ = init
    srv = serve.Server(prec=lbpc.FP32, hbm_budget_bytes=1 << 30, max_chunk=50, clock=FakeClock())
    res = {r.rid: r for r in srv.run(reqs)}
    assert res[1].status == "failed" and res[1].message == "non-physical state" and res[1].steps == 100
    for k in (0, 2, 3):
        assert res[k].status == "ok" and res[k].steps == 300
    assert srv.stats()["failures"] == {"non-physical state": 1}


def test_poisson_stream_is_seeded_and_has_the_requested_rate():
    a = serve.poisson_stream(2000, rate=40.0, seed=3)
    b = serve.poisson_stream(2000, rate=40.0, seed=3)
    assert [(r.kind, r.side, r.steps, r.arrival) for r in a] == [(r.kind, r.side, r.steps, r.arrival) for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert abs(gaps.mean() - 1 / 40.0) < 0.1 / 40.0  # exponential gaps of mean 1/rate
    kinds = [r.kind for r in a]
    assert 0.45 < kinds.count("evaporation") / len(kinds) < 0.55
    assert all(64 <= r.side <= 1024 and 5000 <= r.steps <= 50000 for r in a)


def test_error_that_names_no_instance_propagates(fake):
    """A device error that no single instance owns ends the run instead of looping on the check."""
    orig_check = FakeBatch.check

    def check(self):
        if any(s >= 60 for s in self.steps.values()):
            raise lbpc.LbpcError(lbpc.LBPC_ECUDA, "fake device error")
        orig_check(self)

    fake.check = check
    srv = serve.Server(prec=lbpc.FP32, hbm_budget_bytes=1 << 30, max_chunk=30, clock=FakeClock())
    with pytest.raises(lbpc.LbpcError) as ei:
        srv.run([_req(0, 24, 300, 0.0), _req(1, 24, 300, 0.0)])
    assert ei.value.status == lbpc.LBPC_ECUDA
