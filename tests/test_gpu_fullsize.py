"""Parity at the benchmark's full size (2N = 512, M = 32, in the bench's launch
configuration: graph replay on a stream of its own) on outputs the oracle can
compute one at a time: sampled pair elements G_ab and h_ba (magnitude and phase
against bars from the conditioning of Gamma_a + Gamma_b and Gamma_0 + Delta:
the overlaps of these random states are as small as 1e-40), the energy of the
GPU's (G, h), dGamma of sampled states and their updated Gamma.  Both
arithmetics of the FP64 products are covered: the emulated products (the
library's default and the bench's) with the autotuner (it picks 16 / 16 on
GB300) and with a wider Gauss-Jordan leaf fixed (48 / 16), and the FP64 FMA
products.  A 20-step trajectory compares the two
arithmetics with each other.  At the largest rank (M = 64) on a small chain
the whole pair pass is compared."""
import numpy as np
import pytest

import sgs_inputs as inp
from amplitude_conditioning import dgamma_rtol, lambda_error_bound, overlap_error_bars
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu
RTOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


@pytest.fixture(scope="module")
def large():
    w = inp.LARGE
    p = w.model
    g, lam = inp.initial_state(p.n_modes, w.rank, w.seed, w.parity)
    model = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V)
    return w, p, g, lam, model


VARIANTS = {
    "emulated_gj48": (0, (48, 16)),
    "emulated_autotuned": (0, None),
    "fma_autotuned": (1, None),
}


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_large_workload_sampled_outputs(pkg, large, variant):
    import torch
    w, p, g, lam, model = large
    path, widths = VARIANTS[variant]
    s = pkg.Solver(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, lam, dtau=w.dtau, parity=w.parity,
                   stream=torch.cuda.Stream(), autotune=True, fp64_path=path)
    if widths:
        s.set_panel_widths(*widths)
        assert s.tuning(0)[:2] == widths
    E = s.step(1)[0, 0]                       # graph replay of one step
    G, h = s.pair_matrices()
    g1, lam_g = s.get_state()
    dg = s.derivative()
    s.close()
    rng = np.random.default_rng(0)
    pairs = [(0, 5), (0, 31), (3, 4), (7, 19), (12, 30), (30, 31)]
    for a, b in pairs:
        Go, hbo = orc.pair_elements(model, list(g), a, b)
        # magnitude and phase against bars from the conditioning of the two factorisations
        # they come from (overlap_error_bars); h_ba = conj(G_ab) Wick(Delta) carries both
        mag, ph = overlap_error_bars(g[a], g[b], g[0] if a != 0 else None, orc.transition_matrix(g[a], g[b]), RTOL)
        assert abs(np.log(abs(G[a, b]) / abs(Go))) <= mag, (a, b, mag)
        assert abs(np.angle(G[a, b] / Go)) <= ph, (a, b, ph)
        assert abs(h[b, a] - hbo) <= (mag + ph + RTOL) * abs(hbo), (a, b)
    for a in rng.choice(32, 3, replace=False):
        assert abs(h[a, a] - orc.wick_energy_density(model, g[a])) <= RTOL * abs(h[a, a])
    # the energy and amplitudes of the GPU's (G, h) by the oracle's solve
    Eo, lo = orc.solve_amplitudes(G, h)
    assert abs(E - Eo) <= RTOL * abs(Eo)
    bound = lambda_error_bound(G, h, Eo, lo, G, h)
    assert np.all(np.abs(lam_g - lo) <= 2.0 * bound)
    # dGamma of sampled states from the oracle's equation of motion on the same (G, h, lambda),
    # and the state each one moves to (the exact orthogonal step, then the polar factor)
    mus = [0, 17]
    do = orc.eom(model, list(g), G, h, Eo, lo, mus=mus)
    for mu, d in zip(mus, do):
        rt = dgamma_rtol(bound, lo, mu)
        assert np.abs(dg[mu] - d).max() <= rt * np.abs(d).max(), (mu, rt)
        go = orc.purify(orc.orthogonal_step(g[mu], d, w.dtau))
        assert np.abs(g1[mu] - go).max() <= 1e-9 + w.dtau * rt * np.abs(d).max(), mu
        assert np.abs(g1[mu] @ g1[mu] + np.eye(2 * p.n_modes)).max() < 1e-12


def test_large_trajectory_emulated_against_fma(pkg, large):
    """20 steps at 2N = 512, M = 32 on both arithmetics from the same states:
    the energies agree at the FP64 bar all along."""
    import torch
    w, p, g, lam, _ = large
    out = []
    for path in (0, 1):
        s = pkg.Solver(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, lam, dtau=w.dtau, parity=w.parity,
                       stream=torch.cuda.Stream(), fp64_path=path)
        out.append(s.step(20)[0])
        s.close()
    dev = np.abs(out[0] - out[1]) / np.abs(out[1])
    print(f"20-step energy deviation, emulated vs FMA products: max {dev.max():.3e}, last {dev[-1]:.3e}")
    assert dev.max() <= RTOL


def test_largest_rank_whole_pair_pass(pkg):
    """M = 64 (the largest rank the amplitude solver takes): 2016 pairs."""
    p = inp.AndersonParams(n_bath=6, U=2.0, eps_d=-1.0, V=0.5)        # 2N = 28
    rng = np.random.default_rng(64)
    g = inp.clustered_pure_gammas(p.n_modes, 64, rng, 1, spread=1.5)
    Eo, lo, Go, ho = orc.energy(orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V), list(g))
    for path in (0, 1):
        s = pkg.Solver(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, None, fp64_path=path)
        E = s.energy()[0]
        G, h = s.pair_matrices()
        s.close()
        assert np.abs(G - Go).max() <= RTOL * np.abs(Go).max()
        assert np.abs(h - ho).max() <= RTOL * np.abs(ho).max()
        assert abs(E - Eo) <= 1e-9 * abs(Eo)
