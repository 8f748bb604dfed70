"""The Renyi-2 trace terms (App. B, Eq. S2_SGS) as the CUDA path evaluates them,
on the CPU, against the oracle's form of the paper's Eq. TrArho2_final.

The kernels use the transition operator X_ab = |a><b| / <b|a>, whose two-point
matrix is Delta^{a,b} (Sec. III B): rho_a rho_b = |G_ab|^2 X_ab, a partial trace
keeps the A block, and the trace of two unit-trace Gaussian operators on A is
2^-N_A Pf([[D1, i 1], [-i 1, D2]]).  So, with w_ab = lambda_a conj(lambda_b) G_ba,
  T^{ab}_{cd} = w_ab w_cd 2^-N_A Pf([[Delta^{ab}_A, i 1], [-i 1, Delta^{cd}_A]]),
which must equal the oracle's lambda_a conj(lambda_b) lambda_c conj(lambda_d)
I^{ab}_{cd} / (G_ab G_cd) term by term.  The Pfaffian is taken by a transcription
of the kernel's complex Parlett-Reid (pivot on column k, symmetric interchange of
k + 1 and the pivot row, rank-2 update of the trailing block).  A mistake that
takes Delta^{b,a} for Delta^{a,b} is caught."""
import math

import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc


def parlett_reid_pf(Z):
    Z = Z.astype(complex).copy()
    m = Z.shape[0]
    sign, logm, phase = 1.0, 0.0, 1.0 + 0.0j
    for k in range(0, m - 1, 2):
        col = np.abs(Z[k + 1:, k]) ** 2
        p = k + 1 + int(np.argmax(col))
        if not col.max() > 0.0:
            return 0.0
        if p != k + 1:
            Z[[k + 1, p], :] = Z[[p, k + 1], :]
            Z[:, [k + 1, p]] = Z[:, [p, k + 1]]
            sign = -sign
        piv = Z[k, k + 1]
        logm += math.log(abs(piv))
        phase *= piv / abs(piv)
        tau = Z[k, k + 2:] / piv
        u = Z[k + 2:, k + 1]
        Z[k + 2:, k + 2:] += np.outer(tau, u) - np.outer(u, tau)
    return sign * phase * math.exp(logm)


def delta(gammas, a, b):
    return gammas[a].astype(complex) if a == b else orc.transition_matrix(gammas[a], gammas[b])


def kernel_term(gammas, lam, G, a, b, c, d, NA, conj_slip=False):
    na2 = 2 * NA
    Dab = delta(gammas, b, a) if conj_slip else delta(gammas, a, b)
    Dcd = delta(gammas, c, d)
    I = np.eye(na2)
    Z = np.block([[Dab[:na2, :na2], 1j * I], [-1j * I, Dcd[:na2, :na2]]])
    w_ab = lam[a] * np.conj(lam[b]) * G[b, a]
    w_cd = lam[c] * np.conj(lam[d]) * G[d, c]
    return w_ab * w_cd * 2.0 ** -NA * parlett_reid_pf(Z)


def test_parlett_reid_transcription():
    rng = np.random.default_rng(1)
    for m in (2, 4, 6, 10):
        X = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        A = X - X.T
        assert abs(parlett_reid_pf(A) - orc.pfaffian(A)) < 1e-12 * max(1.0, abs(orc.pfaffian(A)))


@pytest.mark.parametrize("NA", [1, 2])
def test_transition_form_equals_the_papers_form_term_by_term(NA):
    model = orc.anderson_model(2, 2.0, -1.0, 0.5)
    gammas, lam = inp.initial_state(model.N, 3, 4, 1)
    gammas = list(gammas)
    G, h = orc.gram_and_hamiltonian(model, gammas)
    E, lam = orc.solve_amplitudes(G, h)
    M = len(gammas)
    total = 0.0 + 0.0j
    for a in range(M):
        for b in range(M):
            for c in range(M):
                for d in range(M):
                    ref = (lam[a] * np.conj(lam[b]) * lam[c] * np.conj(lam[d])
                           * orc.renyi2_trace_term(gammas[a], gammas[b], gammas[c], gammas[d], NA)
                           / (G[a, b] * G[c, d]))
                    got = kernel_term(gammas, lam, G, a, b, c, d, NA)
                    assert abs(got - ref) < 1e-11 * max(1e-3, abs(ref)), (a, b, c, d)
                    # the symmetry that halves the kernel's count: T^{cd}_{ab} = T^{ab}_{cd}, no conjugate
                    swap = kernel_term(gammas, lam, G, c, d, a, b, NA)
                    assert abs(swap - got) < 1e-12 * max(1e-3, abs(got))
                    total += got
    assert abs(-math.log(total.real) - orc.renyi2(gammas, lam, G, NA)) < 1e-10


def test_conjugate_slip_is_caught():
    model = orc.anderson_model(2, 2.0, -1.0, 0.5)
    gammas, _ = inp.initial_state(model.N, 3, 5, 1)
    gammas = list(gammas)
    G, h = orc.gram_and_hamiltonian(model, gammas)
    E, lam = orc.solve_amplitudes(G, h)
    worst = 0.0
    for a, b, c, d in ((0, 1, 2, 0), (1, 2, 0, 1), (2, 1, 1, 0)):
        ref = (lam[a] * np.conj(lam[b]) * lam[c] * np.conj(lam[d])
               * orc.renyi2_trace_term(gammas[a], gammas[b], gammas[c], gammas[d], 2) / (G[a, b] * G[c, d]))
        bad = kernel_term(gammas, lam, G, a, b, c, d, 2, conj_slip=True)
        worst = max(worst, abs(bad - ref) / abs(ref))
    assert worst > 1e-3
