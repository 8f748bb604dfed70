"""Uneven independent instances advanced together (GPU): one captured graph per
step with one branch per instance.  Each instance of the batch matches the FP64
oracle run on it alone: energies within 1e-10 relative, updated states within
1e-9 (clustered states: order-one amplitudes, so the conditioning widening of
dGamma is negligible)."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def test_uneven_batch_matches_oracle_per_instance(pkg):
    import torch
    ws = inp.batched_workloads(5, seed=21, n_bath=(7, 30), ranks=(2, 3, 5))
    assert len({(w.model.n_bath, w.rank) for w in ws}) > 2        # really uneven
    solver = pkg.Solver(stream=torch.cuda.Stream())
    states = []
    for w in ws:
        p = w.model
        rng = np.random.default_rng(w.seed)
        g = inp.clustered_pure_gammas(p.n_modes, w.rank, rng, w.parity, spread=1.0)
        lam = inp.random_amplitudes(w.rank, rng)
        solver.admit(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels), g, lam, w.dtau,
                     0, 0, w.parity)
        states.append(g)
    E = solver.step(2)
    for k, w in enumerate(ws):
        p = w.model
        model = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels)
        Es, _, go = orc.run(model, list(states[k]), w.dtau, 2)
        assert np.abs(E[k] - Es).max() <= 1e-10 * np.abs(Es).max(), k
        g1, _ = solver.get_state(k)
        assert np.abs(g1 - np.array(go)).max() <= 1e-9, k
    solver.close()
