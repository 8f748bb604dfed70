"""Rank-growth schedule (Sec. III C) and the variance extrapolation of the
energy (Sec. IV A), as host logic over the library's Solver.

The paper starts from a single Gaussian (the mean-field solution), evolves it,
and every ``steps_per_rank`` steps adds one state: a copy of a state of high
amplitude through a random special orthogonal Q close to the identity.  The
library does the copy on the device (``Solver.add_state``); this module only
draws the generator K of Q (a random antisymmetric matrix of a given Frobenius
norm) and runs the schedule.  The energy estimate E* is the intercept of a
linear least-squares fit of E against delta_H^2 over the points with
delta_H^2 below a threshold (2e-5 in the paper), with the intercept's standard
error as its uncertainty.
"""
from __future__ import annotations

import numpy as np


def draw_generator(n: int, norm: float, rng: np.random.Generator) -> np.ndarray:
    """Random antisymmetric n x n K with ||K||_F = norm (exactly antisymmetric)."""
    X = rng.standard_normal((n, n))
    K = X - X.T
    return K * (norm / np.linalg.norm(K))


def grow(solver, slot: int, target_rank: int, steps_per_rank: int, k_norm: float, rng: np.random.Generator,
         with_variance: bool = False):
    """Run the schedule on one slot until it reaches ``target_rank`` and has
    taken ``steps_per_rank`` steps at that rank.  Returns a list with one entry
    per rank: (rank, energies of its steps, (E, delta_H^2) at its end or None)."""
    out = []
    while True:
        M, n = solver.shapes[slot]
        E = solver.step(steps_per_rank)[slot]
        ev = solver.variance(slot) if with_variance else None
        out.append((M, E, ev))
        if M >= target_rank:
            return out
        solver.add_state(draw_generator(n, k_norm, rng), src=-1, slot=slot)


def extrapolate_energy(energies, variances, var_max: float = 2e-5):
    """(E*, sigma): intercept and its standard error of the least-squares line
    E = E* + k delta_H^2 through the points with delta_H^2 < var_max."""
    E = np.asarray(energies, dtype=float)
    v = np.asarray(variances, dtype=float)
    sel = v < var_max
    E, v = E[sel], v[sel]
    m = len(E)
    if m < 3:
        raise ValueError("at least three points below var_max are needed")
    vb, Eb = v.mean(), E.mean()
    sxx = float(((v - vb) ** 2).sum())
    k = float(((v - vb) * (E - Eb)).sum()) / sxx
    e0 = Eb - k * vb
    resid = E - (e0 + k * v)
    s2 = float((resid ** 2).sum()) / (m - 2)
    sigma = float(np.sqrt(s2 * (1.0 / m + vb * vb / sxx)))
    return float(e0), sigma
