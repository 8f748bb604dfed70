"""Parity at the benchmark's full size (2N = 512, M = 32, the bench's launch
configuration: autotuned widths, graph replay) on outputs the oracle can compute
one at a time: sampled pair elements G_ab and h_ba, the energy of the GPU's (G, h),
and dGamma of sampled states.  At the largest rank (M = 64) on a small chain, the
whole pair pass is compared."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu
RTOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def _cond_rtol(lam, mu):
    return RTOL + 50.0 * 2.0 ** -53 * np.abs(lam).max() / max(abs(lam[mu]), 1e-300)


def test_large_workload_sampled_outputs(pkg):
    import torch
    w = inp.LARGE
    p = w.model
    g, lam = inp.initial_state(p.n_modes, w.rank, w.seed, w.parity)
    model = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V)
    s = pkg.Solver(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, lam, dtau=w.dtau, parity=w.parity,
                   stream=torch.cuda.Stream(), autotune=True)
    E = s.step(1)[0, 0]                       # graph replay of one step
    G, h = s.pair_matrices()
    _, lam_g = s.get_state()
    dg = s.derivative()
    s.close()
    rng = np.random.default_rng(0)
    pairs = [(0, 5), (0, 31), (3, 4), (7, 19), (12, 30), (30, 31)]
    for a, b in pairs:
        Go, hbo = orc.pair_elements(model, list(g), a, b)
        assert abs(G[a, b] - Go) <= RTOL * abs(Go), (a, b)
        assert abs(h[b, a] - hbo) <= RTOL * abs(hbo), (a, b)
    for a in rng.choice(32, 3, replace=False):
        assert abs(h[a, a] - orc.wick_energy_density(model, g[a])) <= RTOL * abs(h[a, a])
    # the energy and amplitudes of the GPU's (G, h) by the oracle's solve
    Eo, lo = orc.solve_amplitudes(G, h)
    assert abs(E - Eo) <= RTOL * abs(Eo)
    # dGamma of sampled states from the oracle's equation of motion on the same (G, h, lambda)
    mus = [0, 17]
    do = orc.eom(model, list(g), G, h, Eo, lo, mus=mus)
    for mu, d in zip(mus, do):
        rt = _cond_rtol(lo, mu)
        assert np.abs(dg[mu] - d).max() <= rt * np.abs(d).max(), (mu, rt)


def test_largest_rank_whole_pair_pass(pkg):
    """M = 64 (the largest rank the amplitude solver takes): 2016 pairs."""
    p = inp.AndersonParams(n_bath=6, U=2.0, eps_d=-1.0, V=0.5)        # 2N = 28
    rng = np.random.default_rng(64)
    g = inp.clustered_pure_gammas(p.n_modes, 64, rng, 1, spread=1.5)
    s = pkg.Solver(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, None)
    E = s.energy()[0]
    G, h = s.pair_matrices()
    s.close()
    Eo, lo, Go, ho = orc.energy(orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V), list(g))
    assert np.abs(G - Go).max() <= RTOL * np.abs(Go).max()
    assert np.abs(h - ho).max() <= RTOL * np.abs(ho).max()
    assert abs(E - Eo) <= 1e-9 * abs(Eo)
