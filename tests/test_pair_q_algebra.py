"""The real decomposition of Delta F Delta that the CUDA path's equation of
motion uses (Sec. III B; CPU).  For pure states Gamma_a, Gamma_b
(Gamma^2 = -1), with S = Gamma_a + Gamma_b, D = Gamma_a - Gamma_b, Si = S^-1:

- Delta^{a,b} = (iD - 2) Si = -Si (iD + 2), because S D + D S = 2 (Gamma_a^2 -
  Gamma_b^2) = 0; so Re Delta = -2 Si and Im Delta = D Si = -Si D;
- F = Fr + i Fi with Fr = A + Re Fimp and Fi = Im Fimp, both Fimp parts on the
  rows and columns of the interacting modes only;
- the kernels form Wr = Si Fr Si, V = D Wr, X = V D, L1 = Im[:, imp] Fi,
  L2 = 4 Si[:, imp] Fi, then
  Qr = X + 4 Wr + 2 (L1 Si[imp, :] + Si[:, imp] L1^T),
  Qi = L2 Si[imp, :] - L1 Im[imp, :] - 2 (V - V^T),
  every antisymmetric result as its strictly lower triangle, mirrored.

This test transcribes those steps and requires Qr + i Qi to equal Delta F Delta
with the oracle's transition matrix and Fock matrix.  It also checks that the
identity needs pure states, and that a sign slip in the V term is caught."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc


def skew(M):
    L = np.tril(M, -1)
    return L - L.T


def interacting_modes(model):
    return sorted({i for idx, _ in model.quartic for i in idx} | {i for idx, _ in model.higher for i in idx})


def pair_q(Ga, Gb, A, Fimp, imp, v_slip=False):
    """The kernels' chain for one pair; Fimp: [ni][ni] complex on the interacting modes.
    v_slip: V + V^T in place of V - V^T (a planted mistake)."""
    n = Ga.shape[0]
    S = Ga + Gb
    Si = np.linalg.inv(S)
    D = Ga - Gb
    Im = skew(D @ Si)                                  # Im Delta (antisymmetric product)
    Fr = A.copy()
    Fr[np.ix_(imp, imp)] += Fimp.real
    Fi = Fimp.imag
    T1 = Si @ Fr
    Wr = skew(T1 @ Si)
    V = D @ Wr
    X = skew(V @ D)
    L1 = Im[:, imp] @ Fi
    L2 = 4.0 * (Si[:, imp] @ Fi)
    Qr = skew(X + 4.0 * Wr + 2.0 * (L1 @ Si[imp, :] + Si[:, imp] @ L1.T))
    Qi = skew(L2 @ Si[imp, :] - L1 @ Im[imp, :] - 2.0 * (V + V.T if v_slip else V - V.T))
    return Qr, Qi, Si, Im


def _pair(model, seed, pure=True):
    rng = np.random.default_rng(seed)
    Ga = inp.random_pure_gamma(model.N, rng)
    Gb = inp.random_pure_gamma(model.N, rng)
    if not pure:
        Gb = 0.8 * Gb                                   # a mixed state: Gamma^2 = -0.64
    return Ga, Gb


@pytest.mark.parametrize("n_bath,n_channels,seed", [(3, 1, 1), (5, 1, 2), (2, 2, 3)])
def test_pair_q_equals_delta_f_delta(n_bath, n_channels, seed):
    model = orc.anderson_model(n_bath, 2.0, -1.0, 0.5, n_channels=n_channels)
    imp = interacting_modes(model)
    Ga, Gb = _pair(model, seed)
    Dl = orc.transition_matrix(Ga, Gb)
    F = orc.fock_matrix(model, Dl)
    # the interaction's part of F lives on the interacting modes' block; the rest is A, real
    Fimp = F - model.A
    outside = np.ones(F.shape, bool)
    outside[np.ix_(imp, imp)] = False
    assert np.abs(Fimp[outside]).max() == 0.0
    Qr, Qi, Si, Im = pair_q(Ga, Gb, model.A, Fimp[np.ix_(imp, imp)], imp)
    # Re Delta = -2 Si and Im Delta = D Si
    assert np.abs(Dl.real + 2.0 * Si).max() < 1e-12 * np.abs(Si).max()
    assert np.abs(Dl.imag - Im).max() < 1e-12 * np.abs(Im).max()
    Q = Dl @ F @ Dl
    scale = np.abs(Q).max()
    assert np.abs(Qr - Q.real).max() < 1e-12 * scale
    assert np.abs(Qi - Q.imag).max() < 1e-12 * scale


def test_pair_q_with_higher_terms():
    """A six-Majorana term adds to Fimp on its modes; the decomposition holds unchanged."""
    model = orc.anderson_model(3, 2.0, -1.0, 0.5)
    imp0 = interacting_modes(model)
    extra = tuple(sorted(set(range(8)) - set(imp0)))[:2]
    idx = tuple(imp0[:4]) + extra
    model = orc.MajoranaModel(model.A, model.quartic, model.e_const, [(idx, 0.3)])
    imp = interacting_modes(model)
    Ga, Gb = _pair(model, 4)
    Dl = orc.transition_matrix(Ga, Gb)
    F = orc.fock_matrix(model, Dl)
    Fimp = F - model.A
    Qr, Qi, _, _ = pair_q(Ga, Gb, model.A, Fimp[np.ix_(imp, imp)], imp)
    Q = Dl @ F @ Dl
    scale = np.abs(Q).max()
    assert np.abs(Fimp.imag).max() > 1e-3               # the term makes F complex
    assert np.abs(Qr - Q.real).max() < 1e-12 * scale
    assert np.abs(Qi - Q.imag).max() < 1e-12 * scale


def test_decomposition_needs_pure_states():
    """With a mixed Gamma_b, S D + D S != 0 and Delta is no longer -Si (iD + 2): the chain then
    misses Delta F Delta, which is why the library keeps every state pure (App. A)."""
    model = orc.anderson_model(3, 2.0, -1.0, 0.5)
    imp = interacting_modes(model)
    Ga, Gb = _pair(model, 5, pure=False)
    Dl = orc.transition_matrix(Ga, Gb)
    F = orc.fock_matrix(model, Dl)
    Fimp = F - model.A
    Qr, Qi, _, _ = pair_q(Ga, Gb, model.A, Fimp[np.ix_(imp, imp)], imp)
    Q = Dl @ F @ Dl
    assert np.abs(Qr + 1j * Qi - Q).max() > 1e-3 * np.abs(Q).max()


def test_sign_slip_in_the_v_term_is_caught():
    model = orc.anderson_model(3, 2.0, -1.0, 0.5)
    imp = interacting_modes(model)
    Ga, Gb = _pair(model, 6)
    Dl = orc.transition_matrix(Ga, Gb)
    F = orc.fock_matrix(model, Dl)
    Fimp = F - model.A
    _, Qi, _, _ = pair_q(Ga, Gb, model.A, Fimp[np.ix_(imp, imp)], imp, v_slip=True)
    Q = Dl @ F @ Dl
    assert np.abs(Qi - Q.imag).max() > 1e-3 * np.abs(Q).max()
