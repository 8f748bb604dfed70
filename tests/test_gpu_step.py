"""Whole-step parity of the CUDA path with the FP64 oracle (GPU), on both
arithmetics of the FP64 products (emulated on the tensor cores, the library's
default, and FP64 FMAs).

Bar: energies, G and h within 1e-10 relative; dGamma^mu/ds and the updated
Gamma^mu element by element within 1e-10 of their largest entry, widened by
the conditioning of state mu's amplitude: the decoupling constant c_mu of
Sec. III A divides by lambda_mu, so dGamma^mu moves by |delta lambda_mu| /
|lambda_mu| relative when two solves of h lambda = E G lambda differ by
delta lambda_mu.  That difference is bounded by first-order perturbation
theory from the oracle's (G, h), the two sides' (G, h) and the solves'
backward errors (amplitude_conditioning.py).  Clustered states (order-one
overlaps, order-one amplitudes) make that widening negligible."""
import numpy as np
import pytest

import sgs_inputs as inp
from amplitude_conditioning import dgamma_rtol, lambda_error_bound
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu
RTOL = 1e-10


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def _case(n_bath, U, eps, V, M, seed, parity=1, n_channels=1, t=1.0, mu=0.0, clustered=False):
    p = inp.AndersonParams(n_bath=n_bath, U=U, eps_d=eps, V=V, n_channels=n_channels, t=t, mu=mu)
    if clustered:
        rng = np.random.default_rng(seed)
        g = inp.clustered_pure_gammas(p.n_modes, M, rng, parity, spread=1.0)
        lam = inp.random_amplitudes(M, rng)
    else:
        g, lam = inp.initial_state(p.n_modes, M, seed, parity)
    return p, g, lam


def _solver(pkg, p, g, lam, dtau=0.05, parity=1, cmode=0, fp64_path=0):
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels)
    return pkg.Solver(m, g, lam, dtau=dtau, parity=parity, cmode=cmode, fp64_path=fp64_path)


def _oracle_model(p):
    return orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels)


def _close(a, b, rtol=RTOL):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() <= rtol * scale


PATHS = {"emulated": 0, "fma": 1}


CASES = [
    # (n_bath, U, eps, V, M, seed, parity, channels, clustered)   n = 4 (1 + channels n_bath)
    (15, 2.0, -1.0, 0.5, 4, 1, 1, 1, False),      # small workload: n = 64, M = 4
    (20, 3.0, -1.5, 0.7, 5, 7, 1, 1, False),      # n = 84: ragged tiles
    (3, 2.0, -1.0, 0.5, 3, 11, -1, 2, False),     # two channels, odd parity, n = 28
    (40, 4.0, -2.0, 0.5, 6, 13, 1, 1, False),     # n = 164: several tiles and panels
    (20, 3.0, -1.5, 0.7, 5, 17, 1, 1, True),      # clustered: every amplitude O(1)
    (40, 4.0, -2.0, 0.5, 7, 19, 1, 1, True),
    (10, 8.0, -4.0, 0.6, 6, 23, -1, 2, True),     # two channels, clustered, n = 84
]


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("case", CASES)
def test_pair_matrices_and_energy(pkg, case, path):
    nb, U, e, V, M, seed, par, nc, cl = case
    p, g, lam = _case(nb, U, e, V, M, seed, par, nc, clustered=cl)
    s = _solver(pkg, p, g, lam, parity=par, fp64_path=PATHS[path])
    E = s.energy()[0]
    Gg, hg = s.pair_matrices()
    Eo, lo, Go, ho = orc.energy(_oracle_model(p), list(g))
    assert _close(Gg, Go)
    assert _close(hg, ho)
    assert abs(E - Eo) <= RTOL * abs(Eo)


@pytest.mark.parametrize("path", list(PATHS))
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("cmode", [0, 1])
def test_one_step_matches_oracle(pkg, case, cmode, path):
    nb, U, e, V, M, seed, par, nc, cl = case
    p, g, lam = _case(nb, U, e, V, M, seed, par, nc, clustered=cl)
    s = _solver(pkg, p, g, lam, parity=par, cmode=cmode, fp64_path=PATHS[path])
    E = s.step(1)[0, 0]
    Gg, hg = s.pair_matrices()
    dg = s.derivative()
    g1, lam1 = s.get_state()
    model = _oracle_model(p)
    Eo, lo, Go, ho = orc.energy(model, list(g))
    do = orc.eom(model, list(g), Go, ho, Eo, lo, cmode)
    assert abs(E - Eo) <= RTOL * abs(Eo)
    bound = lambda_error_bound(Go, ho, Eo, lo, Gg, hg)
    assert np.all(np.abs(lam1 - lo) <= 2.0 * bound), np.abs(lam1 - lo) / bound
    for mu in range(M):
        rt = dgamma_rtol(bound, lo, mu)
        assert _close(dg[mu], do[mu], rt), (mu, rt)
        go = orc.purify(orc.orthogonal_step(g[mu], do[mu], 0.05))
        assert np.abs(g1[mu] - go).max() <= 1e-9 + 0.05 * rt * np.abs(do[mu]).max(), mu
        assert np.abs(g1[mu] @ g1[mu] + np.eye(p.n_modes * 2)).max() < 1e-12


def test_trajectory_small_workload(pkg):
    """20 steps of the small plain-FP64 workload against the oracle."""
    w = inp.SMALL
    p = w.model
    g, lam = inp.initial_state(p.n_modes, w.rank, w.seed, w.parity)
    s = _solver(pkg, p, g, lam, dtau=w.dtau)
    Eg = s.step(20)[0]
    Eo, _, go = orc.run(_oracle_model(p), list(g), w.dtau, 20)
    assert np.abs(Eg - Eo).max() <= RTOL * np.abs(Eo).max()
    gg, _ = s.get_state()
    for mu in range(w.rank):
        assert _close(gg[mu], go[mu], 1e-8)


def test_full_small_config_200_steps(pkg):
    """The small workload as configured (2N = 64, M = 4, 200 steps of ds = 0.05,
    plain FP64) against the oracle run of the same 200 steps.  Rounding differences
    of the two implementations grow along the flow only through the smallest
    amplitudes' conditioning; energies stay within 1e-9 relative."""
    w = inp.SMALL
    p = w.model
    g, lam = inp.initial_state(p.n_modes, w.rank, w.seed, w.parity)
    s = _solver(pkg, p, g, lam, dtau=w.dtau)
    Eg = s.step(w.n_steps)[0]
    Eo, _, _ = orc.run(_oracle_model(p), list(g), w.dtau, w.n_steps)
    dev = np.abs(Eg - Eo).max() / np.abs(Eo).max()
    print(f"200-step energy deviation {dev:.3e}, E200 = {Eg[-1]:.12f}")
    assert dev <= 1e-9
    assert np.all(np.diff(Eo) <= 1e-12)            # descent along the whole run


def test_rank_one_and_noninteracting(pkg):
    # M = 1 (GHF) with U = 0: the flow reaches the sum of negative single-particle energies
    p, g, lam = _case(7, 0.0, 0.0, 0.5, 1, 5)
    s = _solver(pkg, p, g, lam, dtau=0.25)
    E = s.step(400)[0]
    h_sp, _ = orc.anderson_chain(7, 0.0, 0.0, 0.5)
    eps = np.linalg.eigvalsh(h_sp)
    assert abs(E[-1] - eps[eps < 0].sum()) < 1e-9
    assert np.all(np.diff(E) <= 1e-12)


def test_checkpoint_resume_is_bitwise(pkg):
    p, g, lam = _case(15, 2.0, -1.0, 0.5, 4, 3)
    s = _solver(pkg, p, g, lam)
    s.step(3)
    gs, ls = s.get_state()
    E1 = s.step(2)[0]
    s.set_state(gs, ls)
    E2 = s.step(2)[0]
    assert np.array_equal(E1, E2)


def test_orthogonal_pair_reports_singular(pkg):
    # two states of different parity have zero overlap: Gamma_a + Gamma_b is singular
    p = inp.AndersonParams(n_bath=3, U=2.0, eps_d=-1.0, V=0.5)
    rng = np.random.default_rng(3)
    g = np.stack([inp.random_pure_gamma(p.n_modes, rng, 1), inp.random_pure_gamma(p.n_modes, rng, -1)])
    s = _solver(pkg, p, g, None)
    with pytest.raises(pkg.SGSError) as e:
        s.energy()
    assert e.value.status == 3


def test_graph_replay_is_bitwise_identical(pkg):
    """The captured-graph step and direct launches run the same kernels."""
    import torch
    p, g, lam = _case(20, 3.0, -1.5, 0.7, 5, 17, clustered=True)
    stream = torch.cuda.Stream()
    out = []
    for graphs in (True, False):
        m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels)
        s = pkg.Solver(m, g, lam, dtau=0.05, stream=stream)
        s.set_graphs(graphs)
        E = s.step(4)[0]
        gg, _ = s.get_state()
        out.append((E, gg))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_library_seeded_states_step(pkg):
    """Admission without gamma0: the library's seeded states equal the test
    generator's, and one step matches the oracle from them."""
    p = inp.AndersonParams(n_bath=20, U=3.0, eps_d=-1.5, V=0.7)
    s = pkg.Solver()
    k = s.admit(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), None, rank=4, seed=77, parity=1)
    g0, lam0 = s.get_state(k)
    gi, li = inp.seeded_states(p.n_modes, 4, 77, 1)
    assert np.abs(g0 - gi).max() < 1e-13 and np.abs(lam0 - li).max() < 1e-15
    E = s.step(1)[k, 0]
    s.close()
    Eo, _, _ = orc.sgs_step(_oracle_model(p), list(gi), 0.05)
    assert abs(E - Eo) <= RTOL * abs(Eo)
