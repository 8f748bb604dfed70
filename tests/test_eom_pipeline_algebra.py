"""The whole equation of motion (Eq. EOM-Gamma3) as the CUDA path composes it,
on the CPU, against the oracle's eom:

- per pair (a < b): S^-1, Im Delta^{a,b} and the interaction's part of
  F^{a,b} on the interacting modes, then Qr, Qi by the real decomposition of
  Delta F Delta (`test_pair_q_algebra.pair_q`);
- the amplitude kernel's per-(mu, beta) coefficients
  (`test_amplitude_algebra.coefficients`);
- the two-pass assembly of the beta != mu terms, with receiver a taking the
  conjugates (`test_eom_assembly_algebra._two_pass`);
- the finish kernel's beta = mu term, 2 (a1x [Gamma, F] + a2x (Gamma F Gamma + F)
  + a3x Gamma) with F = A + the state's interaction block, Gamma F Gamma from
  T2 = F Gamma and Gamma T2.

Every piece is a transcription of a kernel; their composition must give the
oracle's dGamma for every state, for both forms of c_mu."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc
from test_amplitude_algebra import coefficients
from test_eom_assembly_algebra import _two_pass
from test_pair_q_algebra import interacting_modes, pair_q, skew


def own_term(model, Gm, co, imp):
    F = orc.fock_matrix(model, Gm)                     # real: A plus the state's interaction block
    fs = (F - model.A)[np.ix_(imp, imp)]
    Fr = model.A.copy()
    Fr[np.ix_(imp, imp)] += fs
    T2 = Fr @ Gm
    GFG = skew(Gm @ T2)
    gf, fg = Gm @ Fr, Fr @ Gm
    return 2.0 * (co[0] * (gf - fg) + co[2] * (GFG + Fr) + co[4] * Gm)


def composed_eom(model, gammas, cmode, plant_no_conj=False, amplitudes=None):
    """plant_no_conj: a planted mistake, receiver a of each pair takes Delta^{a,b} itself where its
    term needs the conjugate Delta^{b,a}.  amplitudes: (G, h, E, lambda) to use (default: the
    oracle's)."""
    M = len(gammas)
    n = model.n
    imp = interacting_modes(model)
    if amplitudes is None:
        G, h = orc.gram_and_hamiltonian(model, gammas)
        E, lam = orc.solve_amplitudes(G, h)
    else:
        G, h, E, lam = amplitudes
    co3 = coefficients(G, h, E, lam, cmode)
    coef = np.zeros((M, M, 6))
    coef[..., 0::2] = co3.real
    coef[..., 1::2] = co3.imag
    pairs = [(a, b) for a in range(M) for b in range(a + 1, M)]
    si, im, qr, qi, fimp = [], [], [], [], []
    for a, b in pairs:
        Dl = orc.transition_matrix(gammas[a], gammas[b])
        Fimp = (orc.fock_matrix(model, Dl) - model.A)[np.ix_(imp, imp)]
        Qr, Qi, Si, Im = pair_q(gammas[a], gammas[b], model.A, Fimp, imp)
        si.append(Si); im.append(Im); qr.append(Qr); qi.append(Qi)
        fimp.append(np.stack([Fimp.real, Fimp.imag], axis=-1))
    c = dict(n=n, M=M, imp=imp, A=model.A, pairs=pairs, si=si, im=im, qr=qr, qi=qi, fimp=fimp, coef=coef)
    out = []
    for mu in range(M):
        cm = c
        if plant_no_conj:   # the pair listed with mu second: _two_pass then takes no conjugate for mu
            cm = dict(c, pairs=[(b, a) if mu == a else (a, b) for a, b in pairs])
        d = _two_pass(cm, mu) + own_term(model, gammas[mu], coef[mu, mu], imp)
        out.append(skew(d))                             # the kernels store the lower triangle, mirrored
    return out


@pytest.mark.parametrize("cmode", [orc.C_INVERSE, orc.C_PHASE])
@pytest.mark.parametrize("n_bath,n_channels,M,seed", [(3, 1, 4, 1), (2, 2, 3, 2)])
def test_composed_eom_equals_the_oracle(cmode, n_bath, n_channels, M, seed):
    model = orc.anderson_model(n_bath, 2.0, -1.0, 0.5, n_channels=n_channels)
    rng = np.random.default_rng(seed)
    gammas = [inp.random_pure_gamma(model.N, rng) for _ in range(M)]
    G, h = orc.gram_and_hamiltonian(model, gammas)
    E, lam = orc.solve_amplitudes(G, h)
    ref = orc.eom(model, gammas, G, h, E, lam, mode=cmode)
    got = composed_eom(model, gammas, cmode)
    for mu in range(M):
        scale = max(np.abs(ref[mu]).max(), 1e-300)
        assert np.abs(got[mu] - ref[mu]).max() < 1e-10 * scale, mu


def test_relabelling_changes_nothing_and_a_missing_conjugate_is_caught():
    """Swapping two states' labels permutes the result (the pair order (min, max) is a convention);
    receiver a taking Delta^{a,b} instead of its conjugate leaves the oracle."""
    model = orc.anderson_model(3, 2.0, -1.0, 0.5)
    rng = np.random.default_rng(3)
    gammas = [inp.random_pure_gamma(model.N, rng) for _ in range(3)]
    G, h = orc.gram_and_hamiltonian(model, gammas)
    E, lam = orc.solve_amplitudes(G, h)
    ref = orc.eom(model, gammas, G, h, E, lam)
    scale = max(np.abs(r).max() for r in ref)
    swapped = composed_eom(model, [gammas[i] for i in (0, 2, 1)], orc.C_INVERSE)
    assert max(np.abs(swapped[2] - ref[1]).max(), np.abs(swapped[1] - ref[2]).max()) < 1e-10 * scale
    bad = composed_eom(model, gammas, orc.C_INVERSE, plant_no_conj=True)
    assert max(np.abs(g - r).max() for g, r in zip(bad, ref)) > 1e-6 * scale
