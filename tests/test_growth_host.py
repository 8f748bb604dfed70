"""Host logic of the rank-growth schedule and the variance extrapolation
(no GPU): the schedule against a fake solver, the fit against the oracle's."""
import numpy as np

from oracle import sgs_oracle as orc
from paper_2105_01088_gb300 import growth


class _FakeSolver:
    def __init__(self, n):
        self.shapes = [(1, n)]
        self.added = []

    def step(self, k):
        M = self.shapes[0][0]
        return np.full((1, k), -float(M))

    def variance(self, slot):
        return -float(self.shapes[slot][0]), 1.0 / self.shapes[slot][0]

    def add_state(self, K, src=-1, slot=0):
        assert np.array_equal(K, -K.T) and abs(np.linalg.norm(K) - 0.3) < 1e-12 and src == -1
        M, n = self.shapes[slot]
        self.shapes[slot] = (M + 1, n)
        self.added.append(K)


def test_schedule_adds_one_state_per_segment():
    s = _FakeSolver(12)
    out = growth.grow(s, 0, 4, 5, 0.3, np.random.default_rng(1), with_variance=True)
    assert [r for r, _, _ in out] == [1, 2, 3, 4] and len(s.added) == 3
    assert all(len(E) == 5 for _, E, _ in out) and out[-1][2] == (-4.0, 0.25)


def test_extrapolation_matches_oracle_fit():
    rng = np.random.default_rng(5)
    v = rng.uniform(0, 3e-5, 12)
    E = -7.5 + 30.0 * v + rng.normal(0, 1e-7, 12)
    a = growth.extrapolate_energy(E, v)
    b = orc.extrapolate_energy(E, v)
    assert abs(a[0] - b[0]) < 1e-12 and abs(a[1] - b[1]) < 1e-12 * max(1.0, b[1]) + 1e-15
