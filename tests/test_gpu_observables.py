"""Observables of the SGS state on the GPU against the FP64 oracle:
spin-spin C(s) (Eq. Cr), two-channel K(r) (Eq. K2CK) and the Renyi-2
entropy of the impurity plus its first sites (App. B).  Bar: 1e-10 of the
largest value (FP64 throughout)."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def _setup(pkg, n_bath, U, eps, V, M, seed, clustered, parity=1, n_channels=1):
    p = inp.AndersonParams(n_bath=n_bath, U=U, eps_d=eps, V=V, n_channels=n_channels)
    rng = np.random.default_rng(seed)
    if clustered:
        g = inp.clustered_pure_gammas(p.n_modes, M, rng, parity, spread=1.0)
    else:
        g = np.stack([inp.random_pure_gamma(p.n_modes, rng, parity) for _ in range(M)])
    m = pkg.build_anderson(n_bath, U, eps, V, 1.0, 0.0, n_channels)
    s = pkg.Solver(m, g, None, parity=parity)
    model = orc.anderson_model(n_bath, U, eps, V, n_channels=n_channels)
    E, lam, G, h = orc.energy(model, list(g))
    return s, g, lam, G


@pytest.mark.parametrize("clustered", [False, True])
def test_spin_correlator(pkg, clustered):
    s, g, lam, G = _setup(pkg, 15, 2.0, -1.0, 0.5, 4, 7, clustered)
    sites = list(range(0, 9))
    got = s.correlator(pkg.SGS_CORR_SPIN_SPIN, sites)
    ref = orc.spin_correlator(list(g), lam, G, sites)
    assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()


def test_two_channel_correlator(pkg):
    s, g, lam, G = _setup(pkg, 6, 8.0, -4.0, 0.6, 4, 9, True, parity=-1, n_channels=2)
    rs = [1, 2, 3, 4, 5]
    got = s.correlator(pkg.SGS_CORR_TWO_CHANNEL_K, rs)
    ref = orc.two_channel_correlator(list(g), lam, G, rs)
    assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()


@pytest.mark.parametrize("clustered", [False, True])
def test_renyi2(pkg, clustered):
    s, g, lam, G = _setup(pkg, 7, 3.0, -1.5, 0.6, 3, 11, clustered)
    ls = [0, 1, 2, 3]
    got = s.correlator(pkg.SGS_CORR_RENYI2, ls)
    ref = np.array([orc.renyi2(list(g), lam, G, 2 * (1 + l)) for l in ls])
    assert np.abs(got - ref).max() <= TOL * max(1.0, np.abs(ref).max())


def test_renyi2_single_gaussian_full_size(pkg):
    """M = 1 at 2N = 512: S_2 = -sum_j ln[(1 + nu_j^2)/2] over the eigenvalues
    +-i nu_j of Gamma_A (closed form for one Gaussian state)."""
    p = inp.AndersonParams(n_bath=127, U=4.0, eps_d=-2.0, V=0.5)
    g, _ = inp.initial_state(p.n_modes, 1, 5, 1)
    m = pkg.build_anderson(127, 4.0, -2.0, 0.5)
    s = pkg.Solver(m, g)
    ls = [0, 4, 12]
    got = s.correlator(pkg.SGS_CORR_RENYI2, ls)
    for l, v in zip(ls, got):
        GA = g[0][:4 * (1 + l), :4 * (1 + l)]
        nu = np.sort(np.abs(np.linalg.eigvalsh(1j * GA)))[::2]
        assert abs(v + np.sum(np.log((1.0 + nu ** 2) / 2.0))) < 1e-10


def test_observable_arguments_are_checked(pkg):
    s, g, lam, G = _setup(pkg, 3, 2.0, -1.0, 0.5, 2, 3, False)
    with pytest.raises(pkg.SGSError):
        s.correlator(pkg.SGS_CORR_SPIN_SPIN, [4])        # 4 sites: 0..3
    with pytest.raises(pkg.SGSError):
        s.correlator(pkg.SGS_CORR_RENYI2, [4])


@pytest.mark.parametrize("case", [(20, 3.0, -1.5, 0.7, 5, 13, True, 1, 1), (15, 2.0, -1.0, 0.5, 4, 7, False, 1, 1),
                                  (6, 8.0, -4.0, 0.6, 4, 9, True, -1, 2)])
def test_variance(pkg, case):
    """delta_H^2 (Eq. residual): <H^2> within 1e-10 relative of the oracle's,
    so the variance within 1e-10 <H^2> absolute."""
    nb, U, eps, V, M, seed, cl, par, nch = case
    s, g, lam, G = _setup(pkg, nb, U, eps, V, M, seed, cl, parity=par, n_channels=nch)
    E, var = s.variance()
    Eo, vo = orc.variance(orc.anderson_model(nb, U, eps, V, n_channels=nch), list(g))
    assert abs(E - Eo) <= TOL * abs(Eo)
    assert abs(var - vo) <= TOL * (Eo * Eo + abs(vo)) and vo > 0


def test_variance_several_monomials(pkg):
    """A model with three density-density terms, two sharing Majoranas (repeated
    indices in <H4 H4>), passed through the library's general model input."""
    h = np.array([[0.3, 0.0, -1.0, 0.0, 0.0, 0.0], [0.0, -0.2, 0.0, -0.7, 0.0, 0.0],
                  [-1.0, 0.0, 0.1, 0.0, -0.5, 0.0], [0.0, -0.7, 0.0, 0.4, 0.0, -0.6],
                  [0.0, 0.0, -0.5, 0.0, -0.3, 0.0], [0.0, 0.0, 0.0, -0.6, 0.0, 0.2]])
    model = orc.majorana_from_fermions(h, [(0, 1, 2.0), (2, 3, 1.5), (0, 3, 0.8)])
    idx = np.array([k for k, _ in model.quartic], dtype=np.int32)
    val = np.array([v for _, v in model.quartic])
    m = pkg.MajoranaModel(model.A, idx, val, model.e_const)
    rng = np.random.default_rng(17)
    g = inp.clustered_pure_gammas(model.N, 3, rng, 1, spread=1.0)
    s = pkg.Solver(m, g, None)
    E, var = s.variance()
    Eo, vo = orc.variance(model, list(g))
    assert abs(E - Eo) <= TOL * abs(Eo)
    assert abs(var - vo) <= TOL * (Eo * Eo + abs(vo))


def test_renyi2_large_subsystems(pkg):
    """Subsystems past the shared-memory Pfaffian (4(1 + l) > 52) go through the
    batched blocked Pfaffian in chunks; l = 12 is the last shared-memory size,
    and the whole system (l = 16 here) has S_2 = 0."""
    s, g, lam, G = _setup(pkg, 16, 3.0, -1.5, 0.6, 3, 13, True)
    ls = [12, 13, 15, 16]
    got = s.correlator(pkg.SGS_CORR_RENYI2, ls)
    ref = np.array([orc.renyi2(list(g), lam, G, 2 * (1 + l)) for l in ls])
    assert np.abs(got - ref).max() <= TOL * max(1.0, np.abs(ref).max())
    assert abs(got[-1]) < 1e-10
