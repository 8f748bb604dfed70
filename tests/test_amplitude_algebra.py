"""The amplitude solve (Eq. eigLambda, Sec. III A) as the CUDA path runs it (CPU):
a numpy transcription of

- the real symmetric embedding [[Re, -Im], [Im, Re]] of the Hermitian pair (G, h);
- parallel cyclic Jacobi with round-robin pairing (an even count of indices, one
  idle index when m is odd; the rotations of one round are disjoint, applied to
  every row and then every column, and the annihilated entry set to zero);
- canonical orthogonalisation (eigenvalues of G below cut * max dropped), the
  lowest eigenvector, the normalisation lambda^dag G lambda = 1 and the phase that
  makes the largest |lambda_mu| real and positive;
- the coefficients of Eq. (EOM-Gamma3) with z = conj(lt_mu) c_mu lambda_beta:
  a1 = 2i z G_mu,beta, a2 = 2 z G_mu,beta, a3 = -z (h_mu,beta - E G_mu,beta);

against numpy's eigensolver, the oracle's solve_amplitudes and the oracle's
equation of motion."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc


def round_robin(mm, r):
    def pos(j):
        return 0 if j == 0 else ((j - 1 + r) % (mm - 1)) + 1
    out = []
    for i in range(mm // 2):
        p, q = pos(i), pos(mm - 1 - i)
        out.append((min(p, q), max(p, q)))
    return out


def jacobi_sym(A, m, max_rot_residual=None):
    """A: m x m symmetric (modified in place to its diagonal form); returns (V, sweeps)."""
    V = np.eye(m)
    mm = (m + 1) & ~1
    for sweeps in range(60):
        od = A[~np.eye(m, dtype=bool)]
        off = (od * od).sum()
        dg = (np.diag(A) ** 2).sum()
        if off <= 1e-30 * dg or off < 1e-280:
            return V, sweeps
        for r in range(mm - 1):
            rots = []
            for p, q in round_robin(mm, r):
                if q >= m:
                    continue
                apq = A[p, q]
                if abs(apq) <= 1e-300:
                    continue
                th = (A[q, q] - A[p, p]) / (2.0 * apq)
                with np.errstate(over="ignore"):            # th^2 may overflow: then t = 0, as in IEEE
                    t = (1.0 if th >= 0.0 else -1.0) / (abs(th) + np.sqrt(th * th + 1.0))
                c = 1.0 / np.sqrt(t * t + 1.0)
                if t * c != 0.0:                            # a zero rotation is skipped, its entry kept
                    rots.append((p, q, c, t * c))
            for p, q, c, s in rots:
                ap, aq = A[p].copy(), A[q].copy()
                A[p], A[q] = c * ap - s * aq, s * ap + c * aq
            for p, q, c, s in rots:
                ap, aq = A[:, p].copy(), A[:, q].copy()
                A[:, p], A[:, q] = c * ap - s * aq, s * ap + c * aq
                vp, vq = V[:, p].copy(), V[:, q].copy()
                V[:, p], V[:, q] = c * vp - s * vq, s * vp + c * vq
            for p, q, c, s in rots:
                if max_rot_residual is not None:
                    max_rot_residual.append(abs(A[p, q]) / max(np.abs(A).max(), 1e-300))
                A[p, q] = A[q, p] = 0.0
    return V, -1


def embed(H):
    return np.block([[H.real, -H.imag], [H.imag, H.real]])


def amp_solve(G, h, cut=1e-12):
    M = G.shape[0]
    m = 2 * M
    GR, HR = embed(G), embed(h)
    V1, sw = jacobi_sym(GR, m)
    assert sw >= 0
    w = np.diag(GR).copy()
    keep = [j for j in range(m) if w[j] > cut * w.max()]
    XR = V1[:, keep] / np.sqrt(w[keep])
    Hp = XR.T @ (HR @ XR)
    Hp = 0.5 * (Hp + Hp.T)
    V2, sw = jacobi_sym(Hp, len(keep))
    assert sw >= 0
    jm = int(np.argmin(np.diag(Hp)))
    E = Hp[jm, jm]
    lr = XR @ V2[:, jm]
    lam = lr[:M] + 1j * lr[M:]
    lam = lam / np.sqrt(np.real(lam.conj() @ G @ lam))
    j = int(np.argmax(np.abs(lam)))
    lam = lam * (np.conj(lam[j]) / abs(lam[j]))
    return E, lam


def coefficients(G, h, E, lam, cmode):
    lt = G @ lam
    M = len(lam)
    co = np.zeros((M, M, 3), complex)
    for mu in range(M):
        zz = lam[mu] * np.conj(lt[mu])
        az = abs(zz)
        c = 0.0 if az < 1e-300 else (1.0 / zz if cmode == 0 else np.conj(zz) / az)
        for be in range(M):
            z = np.conj(lt[mu]) * c * lam[be]
            co[mu, be] = (2j * z * G[mu, be], 2.0 * z * G[mu, be], -z * (h[mu, be] - E * G[mu, be]))
    return co


@pytest.mark.parametrize("mm", [2, 4, 6, 8, 12, 64])
def test_round_robin_covers_every_pair_once_in_disjoint_rounds(mm):
    seen = []
    for r in range(mm - 1):
        rnd = round_robin(mm, r)
        idx = [i for pq in rnd for i in pq]
        assert sorted(idx) == list(range(mm))          # a round's rotations are disjoint
        seen += rnd
    assert sorted(seen) == sorted((p, q) for p in range(mm) for q in range(p + 1, mm))


@pytest.mark.parametrize("m,seed", [(2, 0), (5, 1), (8, 2), (17, 3), (64, 4)])
def test_jacobi_diagonalises(m, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((m, m))
    A0 = B + B.T
    A = A0.copy()
    res = []
    V, sw = jacobi_sym(A, m, res)
    assert 0 <= sw < 20
    assert np.abs(np.sort(np.diag(A)) - np.linalg.eigvalsh(A0)).max() < 1e-12 * np.abs(A0).max()
    assert np.abs(V.T @ V - np.eye(m)).max() < 1e-13
    assert np.abs(V @ np.diag(np.diag(A)) @ V.T - A0).max() < 1e-12 * np.abs(A0).max()
    # the explicit zeroing removes rounding only
    assert max(res, default=0.0) < 1e-14


def test_embedding_doubles_the_spectrum():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5))
    H = X + X.conj().T
    w = np.linalg.eigvalsh(H)
    we = np.linalg.eigvalsh(embed(H))
    assert np.abs(we - np.repeat(w, 2)).max() < 1e-12


def _states(M, seed, n_bath=3):
    model = orc.anderson_model(n_bath, 2.0, -1.0, 0.5)
    rng = np.random.default_rng(seed)
    gammas = [inp.random_pure_gamma(model.N, rng) for _ in range(M)]
    G, h = orc.gram_and_hamiltonian(model, gammas)
    return model, gammas, G, h


@pytest.mark.parametrize("M,seed", [(1, 0), (3, 1), (6, 2)])
def test_amplitudes_equal_the_oracle(M, seed):
    _, _, G, h = _states(M, seed)
    E, lam = amp_solve(G, h)
    Eo, lamo = orc.solve_amplitudes(G, h)
    assert abs(E - Eo) < 1e-12 * max(1.0, abs(Eo))
    assert np.abs(lam - lamo).max() < 1e-10
    # a generalised eigenpair of (h, G)
    assert np.abs(h @ lam - E * (G @ lam)).max() < 1e-10 * np.abs(h).max()


def test_dependent_states_are_cut():
    """Two equal states make G singular: one direction is dropped and the energy is that of the
    independent states."""
    model = orc.anderson_model(3, 2.0, -1.0, 0.5)
    rng = np.random.default_rng(9)
    g = [inp.random_pure_gamma(model.N, rng) for _ in range(2)]
    G, h = orc.gram_and_hamiltonian(model, [g[0], g[1], g[1]])
    E, _ = amp_solve(G, h)
    G2, h2 = orc.gram_and_hamiltonian(model, g)
    E2, _ = orc.solve_amplitudes(G2, h2)
    assert abs(E - E2) < 1e-9 * abs(E2)


@pytest.mark.parametrize("cmode", [orc.C_INVERSE, orc.C_PHASE])
def test_coefficients_give_the_oracle_equation_of_motion(cmode):
    """2 Re sum_beta (a1 [D, F] + a2 (D F D + F) + a3 D), D = Delta^{beta,mu}, F = F^{beta,mu}
    (Delta^{mu,mu} = Gamma^mu), equals the oracle's dGamma for every state."""
    M = 4
    model, gammas, G, h = _states(M, 11)
    E, lam = amp_solve(G, h)
    co = coefficients(G, h, E, lam, cmode)
    ref = orc.eom(model, gammas, G, h, E, lam, mode=cmode)
    for mu in range(M):
        acc = np.zeros((model.n, model.n), complex)
        for be in range(M):
            D = gammas[mu].astype(complex) if be == mu else orc.transition_matrix(gammas[be], gammas[mu])
            F = orc.fock_matrix(model, D)
            a1, a2, a3 = co[mu, be]
            acc += a1 * (D @ F - F @ D) + a2 * (D @ F @ D + F) + a3 * D
        out = 2.0 * acc.real
        assert np.abs(out - ref[mu]).max() < 1e-10 * max(1.0, np.abs(ref[mu]).max())
