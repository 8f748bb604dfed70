"""Pairs in chunks (bounded memory): an instance whose per-pair buffers hold a
chunk of the pairs runs the pair pass chunk by chunk for (G, h), then again
for the equation of motion, recomputing S^-1 and Im Delta.  Against the same
instance with every pair at once (the same kernels on the same pairs: energies
to 1e-12, states to 1e-10, the order of the sums over pairs aside) and the
oracle, on both FP64 arithmetics and the TF32 form; chunks of one pair, of a
size that does not divide the pair count, and as many as the pairs; and the
device memory the chunked instance holds."""
import numpy as np
import pytest

import sgs_inputs as inp
from amplitude_conditioning import dgamma_rtol, lambda_error_bound
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def _case(M=6):
    p = inp.AndersonParams(n_bath=20, U=3.0, eps_d=-1.5, V=0.7)          # n = 84
    rng = np.random.default_rng(41)
    g = inp.clustered_pure_gammas(p.n_modes, M, rng, 1, spread=1.0)
    lam = inp.random_amplitudes(M, rng)
    return p, g, lam


@pytest.mark.parametrize("precision,path", [(0, 0), (0, 1), (1, 0)])
@pytest.mark.parametrize("chunk", [1, 4, 15])
def test_chunked_step_equals_all_pairs(pkg, chunk, precision, path):
    """FP64: the same sums in another order, energies to 1e-12 and states to 1e-10 over four
    steps.  TF32: the equation of motion is assembled in float (its partial sums round at
    about 6e-8), so one step's dGamma is compared at 1e-5 of its largest entry and the
    trajectory at the TF32 form's stated energy bar against FP64 (2e-4)."""
    p, g, lam = _case()
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    out = []
    for pc in (0, chunk):
        s = pkg.Solver(m, g, lam, dtau=0.05, precision=precision, fp64_path=path, pair_chunk=pc)
        E1 = s.step(1)[0]
        d1 = s.derivative()
        G, h = s.pair_matrices()
        E = np.concatenate([E1, s.step(3)[0]])
        gg, _ = s.get_state()
        out.append((E, gg, G, h, d1, s.bytes_in_use()))
        s.close()
    (E0, g0, G0, h0, d0, b0), (E1, g1, G1, h1, d1, b1) = out
    assert np.abs(G1 - G0).max() <= 1e-13 and np.abs(h1 - h0).max() <= 1e-12 * np.abs(h0).max()
    if precision == 0:
        assert np.abs(E1 - E0).max() <= 1e-12 * np.abs(E0).max()
        assert np.abs(d1 - d0).max() <= 1e-12 * np.abs(d0).max()
        assert np.abs(g1 - g0).max() <= 1e-10
    else:
        assert E1[0] == E0[0]
        assert np.abs(d1 - d0).max() <= 1e-5 * np.abs(d0).max()
        assert np.abs(E1 - E0).max() <= 2e-4 * np.abs(E0).max()
    if chunk < 15:
        assert b1 < b0                            # the per-pair buffers hold a chunk


def test_chunked_step_matches_oracle(pkg):
    p, g, lam = _case()
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    s = pkg.Solver(m, g, lam, dtau=0.05, pair_chunk=4)
    E = s.step(1)[0, 0]
    Gg, hg = s.pair_matrices()
    dg = s.derivative()
    s.close()
    model = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V)
    Eo, lo, Go, ho = orc.energy(model, list(g))
    do = orc.eom(model, list(g), Go, ho, Eo, lo)
    assert abs(E - Eo) <= 1e-10 * abs(Eo)
    bound = lambda_error_bound(Go, ho, Eo, lo, Gg, hg)
    for mu in range(len(g)):
        rt = dgamma_rtol(bound, lo, mu)
        assert np.abs(dg[mu] - do[mu]).max() <= rt * np.abs(do[mu]).max(), mu


def test_chunked_memory_and_refusals(pkg):
    """At 2N = 164, M = 16 (120 pairs) chunks of 8 pairs hold about a tenth of the per-pair
    memory; observables need every pair at once and are refused."""
    p = inp.AndersonParams(n_bath=40, U=4.0, eps_d=-2.0, V=0.5)
    rng = np.random.default_rng(7)
    g = inp.clustered_pure_gammas(p.n_modes, 16, rng, 1, spread=1.0)
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    full = pkg.Solver(m, g, None)
    Ef = full.step(2)[0]
    bf = full.bytes_in_use()
    full.close()
    s = pkg.Solver(m, g, None, pair_chunk=8)
    Ec = s.step(2)[0]
    bc = s.bytes_in_use()
    assert np.abs(Ec - Ef).max() <= 1e-12 * np.abs(Ef).max()
    assert bc < 0.35 * bf
    with pytest.raises(pkg.SGSError) as e:
        s.correlator(pkg.SGS_CORR_SPIN_SPIN, [0, 1])
    assert e.value.status == 1
    with pytest.raises(pkg.SGSError):
        s.variance()
    s.close()
