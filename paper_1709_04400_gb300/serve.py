"""Continuous-batching service for coupled liquid-vapor simulations.

Requests (a droplet-evaporation or heated-wall set-up, its size, radius or strip width, superheat
and step count) arrive over time. A request is admitted as soon as the device arena (the HBM budget
of the service) has room for its state; its populations then stay resident on the device until it
finishes. Every admitted request advances in the same persistent launch as the others
(`lbpc.Batch`). Requests that arrive while others run join between chunks of steps, so their work
overlaps on the device. Results leave as soon as their step count is reached. An instance's
arithmetic does not depend on its neighbours in the batch, so a result is the same alone and in the
mix.

The scheduler here is host-side bookkeeping only: admission (FIFO by arrival, gated by free arena
bytes), the chunk length (the fewest steps any active request still needs, capped), completion and
failure handling. Every step of the physics runs in liblbpc's kernels.
"""

import time
from collections import deque
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import inputs, lbpc, workloads


@dataclass
class Request:
    rid: int
    kind: str  # "evaporation" | "heated_wall"
    side: int  # grid side (square grids)
    steps: int
    size_param: float  # droplet radius (evaporation) or heated-strip width (heated wall)
    superheat: float  # dT / T_c: ring temperature (evaporation) or strip temperature (heated wall)
    arrival: float = 0.0  # seconds after the start of the stream


@dataclass
class Result:
    rid: int
    status: str  # "ok" | "failed"
    arrival: float
    admitted: float
    done: float
    steps: int
    nodes: int
    message: str = ""
    fields: Optional[tuple] = None
    detail: str = ""  # the library's report of a failure (step, node, cause)

    @property
    def time_to_result(self):
        return self.done - self.arrival


def make_case(req: Request, Tc, rho_v, rho_l):
    """Workload dict and initial fields of a request (see workloads)."""
    if req.kind == "evaporation":
        return workloads.droplet_evaporation(Tc, rho_v, rho_l, n=req.side, radius=req.size_param,
                                             dT_ratio=req.superheat)
    if req.kind == "heated_wall":
        # Closed pool (neutral wall) under a vapour cushion of at most 48 rows. An open top lets the
        # buoyancy (rho - rho_ave) g accelerate the vapour out without bound. In a closed pool the cushion
        # must carry a pressure difference of about (rho_ave - rho_v) g H: a half-full pool of side 734 or
        # more takes it past the saturation pressure, and the vapour over the liquid is drawn to vacuum
        # after about 1800 steps. 48 rows keep it under a third of p_sat at every side.
        return workloads.heated_wall(Tc, rho_v, rho_l, nx=req.side, ny=req.side, strip_width=int(req.size_param),
                                     dT_strip_ratio=req.superheat, top="wall", vapour_rows=min(req.side // 2, 48))
    raise ValueError(req.kind)


def poisson_stream(count, rate, seed, side_lo=64, side_hi=1024, steps_lo=5000, steps_hi=50000):
    """Mixed requests with Poisson arrivals (exponential gaps of mean 1/rate seconds): half droplet
    evaporation, half heated wall; side, step count, radius / strip width and superheat drawn from
    the seed."""
    u = inputs.uniform(seed, 6 * count).reshape(count, 6)
    t, out = 0.0, []
    for k in range(count):
        t += -np.log(1.0 - u[k, 0]) / rate
        side = side_lo + int(u[k, 1] * (side_hi - side_lo + 1))
        steps = steps_lo + int(u[k, 2] * (steps_hi - steps_lo + 1))
        if u[k, 3] < 0.5:
            out.append(Request(k, "evaporation", side, steps, (0.15 + 0.15 * u[k, 4]) * side, 0.05 + 0.25 * u[k, 5], t))
        else:
            width = max(4, int(side * (0.03 + 0.05 * u[k, 4])))
            out.append(Request(k, "heated_wall", side, steps, width, 0.1 + 0.2 * u[k, 5], t))
    return out


class Server:
    """One device, one batch, a FIFO of pending requests."""

    def __init__(self, prec=lbpc.FP32, hbm_budget_bytes=8 << 30, max_chunk=256, keep_fields=False,
                 max_instances=4096, clock=time.perf_counter):
        self.prec = prec
        # the served requests wait on their results: their stream goes before bulk work on the same GPU
        self.batch = lbpc.Batch(prec, hbm_budget_bytes, max_instances=max_instances, high_priority=True)
        p0 = lbpc.Params(nx=8, ny=8)
        self.Tc, _ = lbpc.eos_critical(p0)
        self.rho_v, self.rho_l, _ = lbpc.coexistence(p0, 0.86 * self.Tc)
        self.max_chunk = max_chunk
        self.keep_fields = keep_fields
        self.clock = clock
        self.pending = deque()
        self.active = {}  # instance id -> [request, remaining steps, admitted time, nodes]
        self.results: List[Result] = []
        self.node_steps = 0
        self.chunks = 0
        self._head = None  # (request, params, rho, T, bytes) of the head of the queue, built once

    def _prepared(self, req):
        """The head request's initial fields, parameters and arena bytes, built on the host once and kept
        until the request is admitted or rejected (the head may wait many chunks for arena room)."""
        if self._head is None or self._head[0] is not req:
            case, rho, T = make_case(req, self.Tc, self.rho_v, self.rho_l)
            p = lbpc.params_from_case(case, self.prec)
            self._head = (req, p, rho, T, lbpc.Batch.instance_bytes(p))
        return self._head[1:]

    def _admit(self, now):
        while self.pending:
            req = self.pending[0]
            p, rho, T, need = self._prepared(req)
            if need > self.batch.free_bytes() - (1 << 20):  # keep a little room for the work list
                if not self.active:  # nothing will ever free memory for it
                    self.pending.popleft()
                    self.results.append(Result(req.rid, "failed", req.arrival, now, now, 0, p.nx * p.ny,
                                               f"needs {need} bytes, arena has {self.batch.free_bytes()}"))
                    continue
                return
            try:
                i = self.batch.add(p, rho, T)
            except lbpc.LbpcError as e:
                if e.status == lbpc.LBPC_ENOMEM and self.active:
                    return
                self.pending.popleft()
                self.results.append(Result(req.rid, "failed", req.arrival, now, now, 0, p.nx * p.ny, str(e)))
                continue
            self.pending.popleft()
            self.active[i] = [req, req.steps, now, p.nx * p.ny]

    def _retire(self, now, failed_ids=(), detail=""):
        for i in list(self.active):
            req, left, adm, nodes = self.active[i]
            if i in failed_ids:
                self.results.append(Result(req.rid, "failed", req.arrival, adm, now, req.steps - left, nodes,
                                           "non-physical state", detail=detail))
            elif left == 0:
                f = self.batch.fields(i) if self.keep_fields else None
                self.results.append(Result(req.rid, "ok", req.arrival, adm, self.clock() - self.t0, req.steps, nodes,
                                           fields=f))
            else:
                continue
            self.batch.remove(i)
            del self.active[i]

    def run(self, requests: List[Request]):
        """Serve requests whose `arrival` times are seconds after the call; returns the results."""
        todo = deque(sorted(requests, key=lambda r: r.arrival))
        self.t0 = self.clock()
        while todo or self.pending or self.active:
            now = self.clock() - self.t0
            while todo and todo[0].arrival <= now:
                self.pending.append(todo.popleft())
            self._admit(now)
            if not self.active:
                if todo:  # idle until the next arrival
                    time.sleep(max(0.0, min(todo[0].arrival - (self.clock() - self.t0), 0.01)))
                continue
            chunk = min(self.max_chunk, min(v[1] for v in self.active.values()))
            self.batch.step(chunk)
            for v in self.active.values():  # every active instance took the chunk's steps
                v[1] -= chunk
                self.node_steps += chunk * v[3]
            self.chunks += 1
            while True:  # retire failed instances one by one until the check passes
                try:
                    self.batch.check()
                    break
                except lbpc.LbpcError as e:
                    i = getattr(e, "instance", None)
                    if e.status != lbpc.LBPC_ENONPHYS or i not in self.active:
                        raise  # not a per-instance failure: nothing to retire
                    self._retire(self.clock() - self.t0, failed_ids={i}, detail=str(e))
            self._retire(self.clock() - self.t0)
        self.makespan = self.clock() - self.t0
        return self.results

    def stats(self):
        ok = [r for r in self.results if r.status == "ok"]
        kinds = {}
        for r in self.results:
            if r.status != "ok":
                kinds[r.message] = kinds.get(r.message, 0) + 1
        ttr = np.array([r.time_to_result for r in ok]) if ok else np.array([np.nan])
        return dict(requests=len(self.results), ok=len(ok), failed=len(self.results) - len(ok),
                    p50_s=float(np.percentile(ttr, 50)), p99_s=float(np.percentile(ttr, 99)),
                    mean_s=float(np.mean(ttr)), makespan_s=self.makespan,
                    aggregate_mlups=sum(r.nodes * r.steps for r in self.results) / self.makespan / 1e6,
                    chunks=self.chunks, failures=kinds)

    def close(self):
        self.batch.close()
