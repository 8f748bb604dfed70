"""Continuous-batching request loop for impurity solves.

Requests (a model, initial states, amplitudes) arrive over time.  Each one is
admitted as a slot of one resident context as soon as it has arrived and its
device footprint fits the HBM budget (first come, first served), stays on the
device across steps, and is retired once its energy changes by less than
``tol`` in a step (or after ``max_steps``), releasing its memory for waiting
requests.  Every iteration advances all live slots by one step; their work
overlaps on the device (one graph branch per slot).  Slots never interact, so a
solve gives the same result alone and in the mix.

The loop is host logic only; the solver object is the library's Solver (or any
object with admit / retire / step).
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

SGS_ENOMEM = 2
SGS_DEVICE_FAILURES = (3, 4, 5)      # ESINGULAR, ENOTCONV, ETIMEOUT: one slot's solve failed


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    model: object                  # MajoranaModel
    gamma0: np.ndarray
    lambda0: np.ndarray | None = None
    parity: int = 1


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    energy: float
    converged: bool
    energies: list = field(default_factory=list)
    failed: str = ""                  # device-side error that ended the solve, if any

    @property
    def latency(self):
        return self.finished - self.arrival


def latency_stats(results, t_end=None):
    lat = np.array([r.latency for r in results])
    if len(lat) == 0:
        return {"n": 0}
    span = (t_end if t_end is not None else max(r.finished for r in results)) - min(r.arrival for r in results)
    return {"n": len(lat), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "throughput_per_s": len(lat) / span if span > 0 else float("inf"),
            "makespan_s": float(span)}


class ServingLoop:
    """solver: an object with admit(model, gamma0, lambda0, dtau, precision, cmode, parity) -> slot,
    retire(slot) and step(1) -> energies [n_slots, 1] (one per slot ever admitted)."""

    def __init__(self, solver, dtau=0.05, precision=0, cmode=0, tol=1e-8, max_steps=400, clock=time.perf_counter,
                 sleep=time.sleep, keep_energies=False):
        self.solver = solver
        self.dtau, self.precision, self.cmode = dtau, precision, cmode
        self.tol, self.max_steps = tol, max_steps
        self.clock, self.sleep = clock, sleep
        self.keep_energies = keep_energies
        self.rejected = []
        self.failures = []

    def _admit(self, req):
        return self.solver.admit(req.model, req.gamma0, req.lambda0, self.dtau, self.precision, self.cmode,
                                 req.parity)

    def run(self, requests):
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        live = {}        # slot -> [request, admitted time, steps, last energy, energies]
        results = []
        t0 = self.clock()
        while pending or live:
            now = self.clock() - t0
            while pending and pending[0].arrival <= now:
                req = pending[0]
                try:
                    slot = self._admit(req)
                except Exception as e:                      # noqa: BLE001 (status carried on the error)
                    if getattr(e, "status", None) == SGS_ENOMEM:
                        if not live:                         # cannot fit even alone: reject
                            self.rejected.append(req.rid)
                            pending.popleft()
                            continue
                        break                                # wait for a retirement
                    raise
                pending.popleft()
                live[slot] = [req, now, 0, None, []]
            if not live:
                if pending:
                    self.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                continue
            try:
                E = self.solver.step(1)
            except Exception as e:                          # noqa: BLE001 (status carried on the error)
                # device-side failures of some slots: the error lists them and carries the
                # energies of the others, which took the step
                bad = list(getattr(e, "failed", None) or [])
                if not bad and hasattr(self.solver, "failed_instance"):
                    bad = [self.solver.failed_instance()]
                E = getattr(e, "energies", None)
                if (getattr(e, "status", None) not in SGS_DEVICE_FAILURES or not bad
                        or any(x not in live for x in bad)):
                    raise
                now = self.clock() - t0
                for slot in bad:
                    st = live.pop(slot)
                    self.solver.retire(slot)
                    req = st[0]
                    results.append(Result(req.rid, req.arrival, st[1], now, st[2], float("nan"), False, st[4],
                                          str(e)))
                    self.failures.append(req.rid)
                if E is None:                               # no energies for the others: count the step
                    for other in live.values():
                        other[2] += 1
                        other[3] = None
                    continue
            now = self.clock() - t0
            for slot in list(live):
                st = live[slot]
                e = float(E[slot, 0])
                st[2] += 1
                if self.keep_energies:
                    st[4].append(e)
                converged = st[3] is not None and abs(e - st[3]) < self.tol
                st[3] = e
                if converged or st[2] >= self.max_steps:
                    self.solver.retire(slot)
                    req = st[0]
                    results.append(Result(req.rid, req.arrival, st[1], now, st[2], e, converged, st[4]))
                    del live[slot]
        return sorted(results, key=lambda r: r.rid)


def run_sequential(make_solver, requests, dtau=0.05, precision=0, cmode=0, tol=1e-8, max_steps=400,
                   clock=time.perf_counter, sleep=time.sleep):
    """The same solves one at a time, each in a context of its own (the baseline
    a request loop is compared with)."""
    results = []
    t0 = clock()
    for req in sorted(requests, key=lambda r: r.arrival):
        now = clock() - t0
        if now < req.arrival:
            sleep(req.arrival - now)
        start = clock() - t0
        solver = make_solver()
        slot = solver.admit(req.model, req.gamma0, req.lambda0, dtau, precision, cmode, req.parity)
        last, steps, converged, failed, e = None, 0, False, "", float("nan")
        while steps < max_steps:
            try:
                e = float(solver.step(1)[slot, 0])
            except Exception as err:                    # noqa: BLE001 (status carried on the error)
                if getattr(err, "status", None) not in SGS_DEVICE_FAILURES:
                    raise
                failed, e = str(err), float("nan")
                break
            steps += 1
            if last is not None and abs(e - last) < tol:
                converged = True
                break
            last = e
        solver.close()
        results.append(Result(req.rid, req.arrival, start, clock() - t0, steps, e, converged, failed=failed))
    return results
