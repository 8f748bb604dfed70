"""The lattice two-channel Kondo model of Sec. V on the GPU against the FP64
oracle: 24 quartic monomials on 12 Majoranas (impurity and the first site of
each channel), so the Fock matrix's interaction block, the rank-k terms of
the equation of motion and <H4 H4> all run at more than one monomial."""
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


def _setup(pkg, L, J, M, seed):
    import torch
    rng = np.random.default_rng(seed)
    g = inp.clustered_pure_gammas(4 * L, M, rng, 1, spread=1.0)
    lam = inp.random_amplitudes(M, rng)
    s = pkg.Solver(pkg.build_2ck(L, J, 0.5), g, lam, stream=torch.cuda.Stream())
    return s, g, orc.two_channel_kondo_model(L, J, 0.5)


@pytest.mark.parametrize("L,M", [(6, 4), (13, 5)])
def test_kondo_step_matches_oracle(pkg, L, M):
    s, g, model = _setup(pkg, L, 1.4, M, 40 + L)
    E = s.step(1)[0, 0]
    dg = s.derivative()
    g1, _ = s.get_state()
    Eo, lo, Go, ho = orc.energy(model, list(g))
    do = orc.eom(model, list(g), Go, ho, Eo, lo)
    assert abs(E - Eo) <= RTOL * abs(Eo)
    for mu in range(M):
        assert np.abs(dg[mu] - do[mu]).max() <= RTOL * np.abs(do[mu]).max(), mu
        go = orc.purify(orc.orthogonal_step(g[mu], do[mu], 0.05))
        assert np.abs(g1[mu] - go).max() <= 1e-9, mu
    s.close()


def test_kondo_observables_match_oracle(pkg):
    L = 8
    s, g, model = _setup(pkg, L, 1.4, 4, 77)
    rs = list(range(1, L))
    K = s.correlator(pkg.SGS_CORR_TWO_CHANNEL_K, rs)
    E, var = s.variance()
    s.close()
    Eo, lo, Go, _ = orc.energy(model, list(g))
    Ko = orc.two_channel_correlator(list(g), lo, Go, rs)
    assert np.abs(K - Ko).max() <= RTOL * np.abs(Ko).max()
    _, vo = orc.variance(model, list(g))
    assert abs(E - Eo) <= RTOL * abs(Eo)
    assert abs(var - vo) <= RTOL * (Eo * Eo + vo) and vo > 0
