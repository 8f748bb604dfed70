"""Host logic of the continuous-batching loop with a fake solver (CPU)."""
import numpy as np

from paper_2105_01088_gb300.serving import Request, ServingLoop, latency_stats, run_sequential


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 0.0)


class FakeSolver:
    """Energies relax geometrically per slot; each step costs 1 ms per live slot;
    at most `capacity` slots fit the budget."""

    def __init__(self, clock, capacity=2):
        self.clock, self.capacity = clock, capacity
        self.slots, self.live = [], []
        self.log = []

    def admit(self, model, gamma0, lambda0, dtau, precision, cmode, parity):
        if sum(self.live) >= self.capacity:
            e = RuntimeError("over budget")
            e.status = 2
            raise e
        self.slots.append([float(model), 0])
        self.live.append(True)
        self.log.append(("admit", len(self.slots) - 1, self.clock.t))
        return len(self.slots) - 1

    def retire(self, slot):
        self.live[slot] = False
        self.log.append(("retire", slot, self.clock.t))

    def step(self, n):
        E = np.full((len(self.slots), 1), np.nan)
        for i, (target, k) in enumerate(self.slots):
            if self.live[i]:
                self.slots[i][1] = k + 1
                E[i, 0] = target * (1.0 - 0.5 ** (k + 1))
        self.clock.t += 1e-3 * sum(self.live)
        return E

    def close(self):
        pass


def _reqs(arrivals):
    return [Request(i, a, 1.0 + i, None) for i, a in enumerate(arrivals)]


def test_fifo_admission_budget_and_retirement():
    clk = FakeClock()
    s = FakeSolver(clk, capacity=2)
    loop = ServingLoop(s, tol=1e-6, max_steps=100, clock=clk, sleep=clk.sleep)
    res = loop.run(_reqs([0.0, 0.0, 0.0, 0.5]))
    assert [r.rid for r in res] == [0, 1, 2, 3]
    assert all(r.converged for r in res)
    admits = [x for x in s.log if x[0] == "admit"]
    # the third request waits until a slot is retired (budget of two)
    first_retire = min(t for k, _, t in s.log if k == "retire")
    assert admits[2][2] >= first_retire
    # energies converge to each request's own target (no cross talk between slots)
    for r in res:
        assert abs(r.energy - (1.0 + r.rid)) < 1e-5
    st = latency_stats(res)
    assert st["n"] == 4 and st["p99_s"] >= st["p50_s"] > 0


def test_request_too_large_alone_is_rejected():
    clk = FakeClock()
    s = FakeSolver(clk, capacity=0)
    loop = ServingLoop(s, clock=clk, sleep=clk.sleep)
    assert loop.run(_reqs([0.0])) == [] and loop.rejected == [0]


def test_sequential_baseline_serialises():
    clk = FakeClock()
    res = run_sequential(lambda: FakeSolver(clk), _reqs([0.0, 0.0, 0.0]), tol=1e-6, clock=clk, sleep=clk.sleep)
    assert all(res[i].admitted >= res[i - 1].finished for i in range(1, 3))


class FailingSolver(FakeSolver):
    """Slot 1's solve fails on its third step (a device-side error reported for it)."""

    def __init__(self, clock):
        super().__init__(clock, capacity=3)
        self.bad = -1

    def step(self, n):
        if len(self.slots) > 1 and self.live[1] and self.slots[1][1] == 2:
            for i in range(len(self.slots)):
                if self.live[i] and i != 1:
                    self.slots[i][1] += 1
            self.bad = 1
            e = RuntimeError("SGS_ENOTCONV: instance 1: exponential step out of range")
            e.status = 4
            raise e
        self.bad = -1
        return super().step(n)

    def failed_instance(self):
        return self.bad


def test_failed_solve_is_retired_and_reported():
    clk = FakeClock()
    s = FailingSolver(clk)
    loop = ServingLoop(s, tol=1e-6, max_steps=100, clock=clk, sleep=clk.sleep)
    res = loop.run(_reqs([0.0, 0.0, 0.0]))
    assert loop.failures == [1]
    bad = res[1]
    assert bad.failed.startswith("SGS_ENOTCONV") and not bad.converged and np.isnan(bad.energy)
    assert ("retire", 1, bad.finished) in s.log
    for r in (res[0], res[2]):                      # the others finish normally
        assert r.converged and not r.failed and abs(r.energy - (1.0 + r.rid)) < 1e-5


class TwoFailSolver(FakeSolver):
    """Slots 0 and 2 fail in the same step (their second); the error carries the
    other slots' energies of that step, as Solver.step's does."""

    def __init__(self, clock):
        super().__init__(clock, capacity=4)

    def step(self, n):
        if len(self.slots) > 2 and self.live[0] and self.live[2] and self.slots[0][1] == 1:
            E = super().step(n)
            E[[0, 2], 0] = np.nan
            e = RuntimeError("SGS_ESINGULAR: instance 0: ... (and 1 more failed instance(s))")
            e.status = 3
            e.failed = [0, 2]
            e.energies = E
            raise e
        return super().step(n)


def test_two_slots_failing_in_one_step():
    clk = FakeClock()
    s = TwoFailSolver(clk)
    loop = ServingLoop(s, tol=1e-6, max_steps=100, clock=clk, sleep=clk.sleep, keep_energies=True)
    res = loop.run(_reqs([0.0, 0.0, 0.0, 0.0]))
    assert sorted(loop.failures) == [0, 2]
    for r in (res[0], res[2]):
        assert r.failed.startswith("SGS_ESINGULAR") and np.isnan(r.energy)
        assert ("retire", r.rid, r.finished) in s.log
    for r in (res[1], res[3]):
        # the healthy slots keep the energy of the failing step: consecutive energies, one per step
        assert r.converged and not r.failed
        assert len(r.energies) == r.steps
        k = np.arange(1, r.steps + 1)
        assert np.allclose(r.energies, (1.0 + r.rid) * (1.0 - 0.5 ** k))


class FailNoEnergiesSolver(FakeSolver):
    """Slot 1 fails in its third step, and the error carries no energies for the
    others (as when the failure is reported before the energies were read back)."""

    def __init__(self, clock, status=4):
        super().__init__(clock, capacity=4)
        self.status = status

    def step(self, n):
        if len(self.slots) > 1 and self.live[1] and self.slots[1][1] == 2:
            super().step(n)                       # the step ran for every slot
            e = RuntimeError("failed")
            e.status = self.status
            e.failed = [1]
            raise e
        return super().step(n)


def test_failure_without_energies_counts_the_step_for_the_others():
    clk = FakeClock()
    s = FailNoEnergiesSolver(clk)
    loop = ServingLoop(s, tol=1e-6, max_steps=100, clock=clk, sleep=clk.sleep, keep_energies=True)
    res = loop.run(_reqs([0.0, 0.0, 0.0]))
    assert loop.failures == [1] and res[1].failed and res[1].steps == 2
    for r in (res[0], res[2]):
        # one step without an energy: the convergence test restarts from the next energy
        assert r.converged and not r.failed
        assert len(r.energies) == r.steps - 1
        k = np.concatenate([np.arange(1, 3), np.arange(4, r.steps + 1)])
        assert np.allclose(r.energies, (1.0 + r.rid) * (1.0 - 0.5 ** k))


def test_a_failure_that_is_not_a_solve_failure_propagates():
    clk = FakeClock()
    s = FailNoEnergiesSolver(clk, status=6)           # a CUDA runtime error: not one slot's solve
    loop = ServingLoop(s, tol=1e-6, max_steps=100, clock=clk, sleep=clk.sleep)
    try:
        loop.run(_reqs([0.0, 0.0]))
    except RuntimeError as e:
        assert e.status == 6
    else:
        raise AssertionError("the error was swallowed")


def test_sequential_baseline_reports_a_failed_solve_and_goes_on():
    clk = FakeClock()

    class OneShot(FakeSolver):
        calls = 0

        def step(self, n):
            OneShot.calls += 1
            if OneShot.calls == 3:
                e = RuntimeError("SGS_ENOTCONV: amplitudes")
                e.status = 4
                raise e
            return super().step(n)

    res = run_sequential(lambda: OneShot(clk), _reqs([0.0, 0.0]), tol=1e-6, max_steps=100, clock=clk,
                         sleep=clk.sleep)
    assert res[0].failed.startswith("SGS_ENOTCONV") and np.isnan(res[0].energy) and res[0].steps == 2
    assert res[1].converged and not res[1].failed
