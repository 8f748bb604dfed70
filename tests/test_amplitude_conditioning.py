"""The first-order amplitude sensitivity behind the dGamma tolerances (CPU):
perturbing (G, h) and re-solving with the oracle moves lambda as the formula of
tests/amplitude_conditioning.py predicts, and never by more than its bound."""
import numpy as np

import sgs_inputs as inp
from amplitude_conditioning import amplitude_sensitivity, lambda_error_bound
from oracle import sgs_oracle as orc


def _problem(rng, M, small_amplitudes):
    """A Hermitian positive G (unit diagonal) and Hermitian h whose lowest
    solution has, if asked, amplitudes down to ~1e-10 of the largest."""
    A = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    G = A @ A.conj().T / M + np.eye(M)
    d = np.sqrt(np.real(np.diag(G)))
    G = G / np.outer(d, d)
    H = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    h = 0.5 * (H + H.conj().T)
    if small_amplitudes:
        # make state 0 carry the ground state almost alone: h = G-weighted projector
        v = np.zeros(M, complex)
        v[0] = 1.0
        h = h * 1e-3 - 5.0 * np.outer(G @ v, (G @ v).conj())
    return G, h


def _gauge(dl, lam):
    """Remove the global-phase part the solver's gauge (largest |lambda| real) fixes."""
    p = int(np.argmax(np.abs(lam)))
    return dl - 1j * np.imag(dl[p] / lam[p]) * lam


def test_first_order_prediction_and_bound():
    rng = np.random.default_rng(5)
    for M, small in ((6, False), (6, True), (12, False), (12, True)):
        G, h = _problem(rng, M, small)
        E, lam = orc.solve_amplitudes(G, h)
        S = amplitude_sensitivity(G, h)
        for eps in (1e-7, 1e-9):
            dG = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
            dG = eps * 0.5 * (dG + dG.conj().T)
            dh = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
            dh = eps * 0.5 * (dh + dh.conj().T)
            E2, lam2 = orc.solve_amplitudes(G + dG, h + dh)
            pred = -S @ ((dh - E * dG) @ lam) - 0.5 * np.real(lam.conj() @ dG @ lam) * lam
            pred = _gauge(pred, lam)
            act = lam2 - lam
            # second-order agreement, state by state
            assert np.all(np.abs(act - pred) <= 1e-4 * np.abs(act).max() + 1e-3 * np.abs(act)), (M, small, eps)
            bound = lambda_error_bound(G, h, E, lam, G + dG, h + dh)
            assert np.all(np.abs(act) <= bound), (M, small, eps)


def test_bound_catches_a_dropped_term():
    """The bound is not loose by orders: dropping the resolvent (S = 0) or the
    perturbation term leaves a real perturbation unexplained."""
    rng = np.random.default_rng(9)
    G, h = _problem(rng, 8, True)
    E, lam = orc.solve_amplitudes(G, h)
    dh = 1e-8 * np.diag(rng.standard_normal(8))
    _, lam2 = orc.solve_amplitudes(G, h + dh)
    act = np.abs(lam2 - lam)
    bound = lambda_error_bound(G, h, E, lam, G, h + dh)
    assert np.all(act <= bound)
    assert act.max() > 1e-3 * bound.max()


def test_overlap_error_bars_bound_perturbed_factorisations():
    """The bars of overlap_error_bars hold for inputs perturbed by the backward error they
    assume (n u |X|_2, random direction) and fail for a perturbation 1e4 times larger in
    the worst direction: the first-order log-determinant identity is what they rest on."""
    from amplitude_conditioning import U, overlap_error_bars
    rng = np.random.default_rng(8)
    n_modes = 12
    g = [inp.random_pure_gamma(n_modes, rng, 1) for _ in range(3)]
    D = orc.transition_matrix(g[1], g[2])
    mag, ph = overlap_error_bars(g[1], g[2], g[0], D, rtol=0.0)
    S = g[1] + g[2]
    Y = g[0] + D
    n = S.shape[0]
    for _ in range(20):
        E = rng.standard_normal((n, n))
        E = E - E.T
        dS = E * (n * U * np.linalg.norm(S, 2) / np.linalg.norm(E, 2))
        d_mag = abs(0.5 * (np.linalg.slogdet(S + dS)[1] - np.linalg.slogdet(S)[1]))
        assert d_mag <= mag
        F = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        F = F - F.T
        dY = F * (n * U * np.linalg.norm(Y, 2) / np.linalg.norm(F, 2))
        p0, _ = orc.pfaffian_log(Y)
        p1, _ = orc.pfaffian_log(Y + dY)
        assert abs(np.angle(p1 / p0)) <= ph
    # along the smallest singular direction a 1e4 times larger perturbation breaks the bar
    Us, sv, Vt = np.linalg.svd(S)
    k = np.argmin(sv)
    P = np.outer(Us[:, k], Vt[k])
    dS = (P - P.T) * (1e4 * n * U * sv[0] * np.sum(1.0 / sv))
    assert abs(0.5 * (np.linalg.slogdet(S + dS)[1] - np.linalg.slogdet(S)[1])) > mag
