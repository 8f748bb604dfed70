"""Pair-sharded imaginary-time step: one SGS problem over several ranks.

The M(M-1)/2 state pairs of a step are independent units (Sec. III C: the
overlaps, transition matrices, Hamiltonian elements and the pairs' terms of
the equation of motion), so each rank evaluates a share of them.  Pair p in
the order (0, 1), (0, 2), ..., (M - 2, M - 1) belongs to rank p mod world, and
the own (beta = mu) terms of state mu to rank mu mod world.  Every rank holds
all M covariance matrices.  One step:

    1. pair pass over the rank's pairs     -> its share of (G, h)    [M x M complex, twice]
       sum over ranks (all-reduce)          -> (G, h)
    2. amplitude solve (Eq. eigLambda; the same on every rank), equation of
       motion of the rank's pairs and own states -> its share of dGamma/ds   [M x 2N x 2N]
       sum over ranks (all-reduce)          -> dGamma/ds
    3. orthogonal update and re-purification of every state (App. A; the same
       on every rank, so the states stay equal without a third exchange).

An all-reduce moves the bytes of a reduce-scatter plus an all-gather, so
summing dGamma/ds everywhere costs the exchange of reducing it to owners and
gathering the updated states; the price is that every rank runs the per-state
update.  The library does stages 1-3 (sgs_shard_pairs / eom / update); this
module is the host-side loop that makes the two sums with torch.distributed.
Any backend object with the three stage methods can be driven, which lets the
partition and the reductions be tested on CPU ranks (gloo).
"""
from __future__ import annotations

import numpy as np


def pair_list(M):
    """Pairs (a, b), a < b, in the library's order."""
    return [(a, b) for a in range(M) for b in range(a + 1, M)]


def local_pairs(M, rank, world):
    """The pairs rank holds: index in pair_list(M) equal to rank modulo world."""
    return [ab for p, ab in enumerate(pair_list(M)) if p % world == rank]


def own_states(M, rank, world):
    """The states whose own (beta = mu) terms rank adds."""
    return [mu for mu in range(M) if mu % world == rank]


def _all_reduce(dist, t, group):
    """Sum over ranks in place.  gloo reduces host tensors: a device tensor is staged
    through host memory on that backend."""
    if t.is_cuda and dist.get_backend(group) == "gloo":
        h = t.cpu()
        dist.all_reduce(h, group=group)
        t.copy_(h)
    else:
        dist.all_reduce(t, group=group)


class LibraryShard:
    """The library's stage calls for one rank: a Solver slot admitted with
    shard=(rank, world), exchange buffers on the current CUDA device."""

    def __init__(self, solver, slot=0):
        import torch
        self.torch = torch
        self.solver, self.slot = solver, slot
        M, n = solver.shapes[slot]
        self.gh = torch.zeros(4 * M * M, dtype=torch.float64, device="cuda")
        self.dg = torch.zeros(M * n * n, dtype=torch.float64, device="cuda")

    def pairs(self):
        self.solver.shard_pairs(self.gh.data_ptr(), self.slot)
        return self.gh

    def eom(self, gh):
        self.torch.cuda.synchronize()          # the sum over ranks ran on torch's stream
        E = self.solver.shard_eom(gh.data_ptr(), self.dg.data_ptr(), self.slot)
        return E, self.dg

    def update(self, dg):
        self.torch.cuda.synchronize()
        self.solver.shard_update(dg.data_ptr(), self.slot)


class ShardedStep:
    """Drives a backend through the step with the two sums over the ranks of `group`."""

    def __init__(self, backend, group=None):
        import torch.distributed as dist
        self.dist, self.backend, self.group = dist, backend, group

    def step(self, n_steps=1):
        """n_steps steps; returns the energy at the start of each (numpy array)."""
        E = np.zeros(n_steps)
        for k in range(n_steps):
            gh = self.backend.pairs()
            _all_reduce(self.dist, gh, self.group)
            E[k], dg = self.backend.eom(gh)
            _all_reduce(self.dist, dg, self.group)
            self.backend.update(dg)
        return E
