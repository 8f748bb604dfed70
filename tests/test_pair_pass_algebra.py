"""The pair pass (Sec. II B-C, Eq. eigLambda) as the CUDA path composes it, on
the CPU, against the oracle's Gram and Hamiltonian matrices:

- |G_ab| from log|det S|, S = Gamma_a + Gamma_b:
  log|G_ab| = (-N log 2 + log|det S| / 2) / 2;
- the phase of G_ab, for a != 0, from parity Pf(Y) with Y = Gamma_0 - 2 S^-1 +
  i Im Delta^{a,b}, the Pfaffian taken by the blocked upper-triangle
  Parlett-Reid transcription (`test_pf_upper_algebra.blocked_pfaffian`); the
  oracle multiplies by Pf(Gamma_0) instead, which is the parity for a pure state
  (Gamma_0 = O J O^T with det O = parity);
- h_ba = conj(G_ab) times the Wick energy density of Delta^{a,b}, and the
  states' diagonal h_aa from Gamma_a.

The composition must give the oracle's (G, h) for both parities; taking the
parity factor away is caught for odd parity."""
import math

import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc
from test_pair_q_algebra import skew
from test_pf_upper_algebra import blocked_pfaffian


def composed_gh(model, gammas, parity, bs=3, use_parity=True):
    M, N = len(gammas), model.N
    G = np.eye(M, dtype=complex)
    h = np.zeros((M, M), dtype=complex)
    for a in range(M):
        h[a, a] = orc.wick_energy_density(model, gammas[a])
    for a in range(M):
        for b in range(a + 1, M):
            S = gammas[a] + gammas[b]
            _, ld = np.linalg.slogdet(S)
            mag = math.exp(0.5 * (-N * math.log(2.0) + 0.5 * ld))
            Si = np.linalg.inv(S)
            Im = skew((gammas[a] - gammas[b]) @ Si)
            Dl = -2.0 * Si + 1j * Im
            ph = 1.0 + 0.0j
            if a != 0:
                pf = blocked_pfaffian(gammas[0] + Dl, bs)
                ph = (parity if use_parity else 1) * pf / abs(pf)
            gab = mag * ph
            G[a, b], G[b, a] = gab, np.conj(gab)
            h[b, a] = np.conj(gab) * orc.wick_energy_density(model, Dl)
            h[a, b] = np.conj(h[b, a])
    return G, h


@pytest.mark.parametrize("parity", [1, -1])
@pytest.mark.parametrize("n_bath,n_channels,M,seed", [(3, 1, 5, 1), (2, 2, 4, 2)])
def test_composed_pair_pass_equals_the_oracle(parity, n_bath, n_channels, M, seed):
    model = orc.anderson_model(n_bath, 2.0, -1.0, 0.5, n_channels=n_channels)
    gammas, _ = inp.initial_state(model.N, M, seed, parity)
    gammas = list(gammas)
    # the shortcut's premise: Pf(Gamma_0) is the parity
    assert abs(orc.pfaffian(gammas[0]) - parity) < 1e-12
    G, h = composed_gh(model, gammas, parity)
    Go, ho = orc.gram_and_hamiltonian(model, gammas)
    assert np.abs(G - Go).max() < 1e-11 * np.abs(Go).max()
    assert np.abs(h - ho).max() < 1e-11 * np.abs(ho).max()


def test_missing_parity_factor_is_caught():
    model = orc.anderson_model(3, 2.0, -1.0, 0.5)
    gammas, _ = inp.initial_state(model.N, 4, 5, -1)
    gammas = list(gammas)
    G, _ = composed_gh(model, gammas, -1, use_parity=False)
    Go, _ = orc.gram_and_hamiltonian(model, gammas)
    assert np.abs(G - Go).max() > 1e-3 * np.abs(Go).max()
