"""Interaction terms of six and eight Majoranas (Sec. II A allows them; the
energy of a term is the Pfaffian of the transition matrix's sub-block on its
indices and its share of the Fock matrix the derivative of that Pfaffian) on
the GPU against the oracle, whose handling of them is pinned against Fock
space (tests/test_oracle_pins.py): G, h and E at 1e-10, dGamma and the next
state at the FP64 bars, a short trajectory, both arithmetics of the FP64
products."""
import numpy as np
import pytest

import sgs_inputs as inp
from amplitude_conditioning import dgamma_rtol, lambda_error_bound
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu
RTOL = 1e-10
HIGHER = [((5, 0, 3, 6, 1, 2), 0.37), ((7, 1, 2, 4, 0, 6, 3, 5), -0.21), ((2, 7, 4, 1, 6, 0), -0.15)]


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def _models(pkg, p):
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V).with_higher(HIGHER)
    base = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V)
    return m, orc.MajoranaModel(base.A, base.quartic, base.e_const, HIGHER)


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("clustered", [True, False])
def test_step_with_higher_terms(pkg, path, clustered):
    p = inp.AndersonParams(n_bath=20, U=3.0, eps_d=-1.5, V=0.7)          # n = 84
    if clustered:
        rng = np.random.default_rng(29)
        g = inp.clustered_pure_gammas(p.n_modes, 5, rng, 1, spread=1.0)
        lam = inp.random_amplitudes(5, rng)
    else:
        g, lam = inp.initial_state(p.n_modes, 5, 31, 1)
    mg, mo = _models(pkg, p)
    s = pkg.Solver(mg, g, lam, dtau=0.05, fp64_path=path)
    E = s.step(1)[0, 0]
    Gg, hg = s.pair_matrices()
    dg = s.derivative()
    g1, lam1 = s.get_state()
    s.close()
    Eo, lo, Go, ho = orc.energy(mo, list(g))
    assert abs(E - Eo) <= RTOL * abs(Eo)
    assert np.abs(Gg - Go).max() <= RTOL * np.abs(Go).max()
    assert np.abs(hg - ho).max() <= RTOL * np.abs(ho).max()
    # the terms matter at this bar
    _, _, _, h0 = orc.energy(orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V), list(g))
    assert np.abs(ho - h0).max() > 1e4 * RTOL * np.abs(ho).max()
    do = orc.eom(mo, list(g), Go, ho, Eo, lo)
    bound = lambda_error_bound(Go, ho, Eo, lo, Gg, hg)
    for mu in range(len(g)):
        rt = dgamma_rtol(bound, lo, mu)
        assert np.abs(dg[mu] - do[mu]).max() <= rt * np.abs(do[mu]).max(), (mu, rt)
        go = orc.purify(orc.orthogonal_step(g[mu], do[mu], 0.05))
        assert np.abs(g1[mu] - go).max() <= 1e-9 + 0.05 * rt * np.abs(do[mu]).max(), mu


def test_trajectory_with_higher_terms(pkg):
    p = inp.AndersonParams(n_bath=15, U=2.0, eps_d=-1.0, V=0.5)          # n = 64
    rng = np.random.default_rng(3)
    g = inp.clustered_pure_gammas(p.n_modes, 4, rng, 1, spread=1.0)
    mg, mo = _models(pkg, p)
    s = pkg.Solver(mg, g, None, dtau=0.05)
    Eg = s.step(10)[0]
    s.close()
    Eo, _, _ = orc.run(mo, list(g), 0.05, 10)
    assert np.abs(Eg - Eo).max() <= RTOL * np.abs(Eo).max()


def test_higher_terms_rejected_where_unsupported(pkg):
    p = inp.AndersonParams(n_bath=6, U=2.0, eps_d=-1.0, V=0.5)
    g, lam = inp.initial_state(p.n_modes, 2, 5, 1)
    mg, _ = _models(pkg, p)
    s = pkg.Solver(mg, g, lam)
    with pytest.raises(pkg.SGSError) as e:
        s.variance()
    assert e.value.status == 1
    s.close()
    bad = mg.with_higher([((0, 1, 2, 3, 4, 4), 1.0)])              # repeated index
    with pytest.raises(pkg.SGSError) as e:
        pkg.Solver(bad, g, lam)
    assert e.value.status == 1
    odd = mg.with_higher([((0, 1, 2, 3, 4), 1.0)])                 # five Majoranas
    with pytest.raises(pkg.SGSError) as e:
        pkg.Solver(odd, g, lam)
    assert e.value.status == 1
