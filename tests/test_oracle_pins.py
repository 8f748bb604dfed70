"""Pins of the FP64 oracle against things other than itself: explicit
Fock-space vectors, exact diagonalisation, closed forms and identities stated
in the paper.  CPU only."""
import math

import numpy as np
import pytest

import fock
import sgs_inputs as inp
from oracle import sgs_oracle as orc


def _rng(seed):
    return np.random.default_rng(seed)


def _fock_operator(model):
    """The oracle's Majorana-form Hamiltonian as a Fock operator."""
    N = model.N
    c = fock.majoranas(N)
    H = model.e_const * fock.sp.identity(2 ** N, dtype=np.complex128, format="csr")
    for k in range(model.n):
        for l in range(model.n):
            if model.A[k, l] != 0.0:
                H = H + (1j * model.A[k, l]) * (c[k] @ c[l])
    for (k, l, p, q), v in model.quartic:
        H = H + v * (c[k] @ c[l] @ c[p] @ c[q])
    for idx, v in model.higher:
        r = len(idx) // 2
        prod = c[idx[0]]
        for x in idx[1:]:
            prod = prod @ c[x]
        H = H + (v * (1j ** (r % 2))) * prod
    return H.tocsr()


def _higher_model():
    """A two-site Anderson model (N = 4 modes) plus one term of six and one of eight
    Majoranas in scrambled index orders (Sec. II A: interaction terms of more than
    four Majoranas)."""
    base = orc.anderson_model(1, 2.0, -1.0, 0.5)
    higher = [((5, 0, 3, 6, 1, 2), 0.37), ((7, 1, 2, 4, 0, 6, 3, 5), -0.21), ((2, 7, 4, 1, 6, 0), -0.15)]
    return orc.MajoranaModel(base.A, base.quartic, base.e_const, higher)


# ---------------------------------------------------------------- model (Sec. II A, IV)

@pytest.mark.parametrize("n_bath,n_channels", [(1, 1), (2, 1), (1, 2)])
def test_majorana_form_equals_fermion_hamiltonian(n_bath, n_channels):
    rng = _rng(10 + n_bath + 7 * n_channels)
    U, eps, V, t, mu = rng.uniform(0.5, 3.0), rng.uniform(-2, 0), rng.uniform(0.2, 1), rng.uniform(0.5, 1.5), rng.uniform(-0.3, 0.3)
    model = orc.anderson_model(n_bath, U, eps, V, t, mu, n_channels)
    Hf = fock.hamiltonian_anderson(n_bath, U, eps, V, t, mu, n_channels)
    Hm = _fock_operator(model)
    assert abs(Hf - Hm).max() < 1e-13


def test_vacuum_and_parity_convention():
    # vacuum has Gamma = J and Pf = +1; one occupied mode flips the parity
    N = 3
    J = inp.vacuum_gamma(N)
    vac = np.zeros(2 ** N, complex)
    vac[0] = 1
    assert np.allclose(fock.covariance_of(vac), J)
    a = fock.annihilators(N)
    one = a[1].conj().T @ vac
    G1 = fock.covariance_of(one)
    assert orc.pfaffian(J) == pytest.approx(1.0)
    assert orc.pfaffian(G1) == pytest.approx(-1.0)


# ---------------------------------------------------------------- Pfaffian

def test_pfaffian_closed_forms():
    rng = _rng(3)
    # 4x4 closed form
    a = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    A = np.zeros((4, 4), complex)
    A[0, 1], A[0, 2], A[0, 3], A[1, 2], A[1, 3], A[2, 3] = a
    A = A - A.T
    ref = A[0, 1] * A[2, 3] - A[0, 2] * A[1, 3] + A[0, 3] * A[1, 2]
    assert abs(orc.pfaffian(A) - ref) < 1e-13
    # block diagonal
    vals = rng.standard_normal(5)
    B = np.zeros((10, 10))
    for j, v in enumerate(vals):
        B[2 * j, 2 * j + 1], B[2 * j + 1, 2 * j] = v, -v
    assert orc.pfaffian(B) == pytest.approx(np.prod(vals), rel=1e-13)
    for n in (6, 12, 20):
        X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        X = X - X.T
        p = orc.pfaffian(X)
        assert abs(p * p - np.linalg.det(X)) < 1e-10 * abs(np.linalg.det(X))
        # Pf(B X B^T) = det(B) Pf(X): fixes the sign, not only the square
        Bm = rng.standard_normal((n, n))
        assert abs(orc.pfaffian(Bm @ X @ Bm.T) - np.linalg.det(Bm) * p) < 1e-9 * abs(np.linalg.det(Bm) * p)


def _pf_by_matchings(A):
    """The definition: the sum over perfect matchings of {0..n-1}, each the product of
    A[i, j] over its pairs (i < j) with the sign of the permutation (i1 j1 i2 j2 ...)."""
    n = A.shape[0]

    def rec(rest):
        if not rest:
            return 1.0
        i, tot = rest[0], 0.0
        for pos in range(1, len(rest)):
            j = rest[pos]
            # moving j next to i crosses pos - 1 indices
            tot += (-1) ** (pos - 1) * A[i, j] * rec(rest[1:pos] + rest[pos + 1:])
        return tot

    return rec(list(range(n)))


def test_pfaffian_equals_the_sum_over_perfect_matchings():
    rng = _rng(4)
    for n in (2, 4, 6, 8):
        X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        X = X - X.T
        ref = _pf_by_matchings(X)
        assert abs(orc.pfaffian(X) - ref) < 1e-12 * max(1.0, abs(ref))
        phase, logmag = orc.pfaffian_log(X)
        assert abs(phase * np.exp(logmag) - ref) < 1e-12 * max(1.0, abs(ref))


# ---------------------------------------------------------------- pair quantities vs Fock

def _states(N, M, seed, parity=1):
    rng = _rng(seed)
    gammas = [inp.random_pure_gamma(N, rng, parity) for _ in range(M)]
    ref = fock.gaussian_vector(gammas[0])
    vecs = [fock.gaussian_vector(g, ref) for g in gammas]
    return gammas, vecs


@pytest.mark.parametrize("parity", [1, -1])
def test_gram_and_h_match_fock(parity):
    model = orc.anderson_model(1, 2.0, -1.0, 0.5)         # 2 sites, N = 4 modes
    gammas, vecs = _states(4, 4, 21 + parity, parity)
    for g, v in zip(gammas, vecs):
        assert np.allclose(fock.covariance_of(v), g, atol=1e-12)
    G, h = orc.gram_and_hamiltonian(model, gammas)
    H = fock.hamiltonian_anderson(1, 2.0, -1.0, 0.5)
    assert np.abs(G - fock.gram(vecs)).max() < 1e-12
    assert np.abs(h - fock.hmat(vecs, H)).max() < 1e-12
    # G Hermitian, positive definite, gauge: G_0mu > 0
    assert np.allclose(G, G.conj().T)
    assert np.linalg.eigvalsh(G).min() > 0
    assert np.all(np.abs(G[0].imag) < 1e-15) and np.all(G[0].real > 0)


def test_transition_matrix_two_and_four_point():
    gammas, vecs = _states(3, 2, 5)
    N, n = 3, 6
    c = fock.majoranas(N)
    a, b = 0, 1
    D = orc.transition_matrix(gammas[a], gammas[b])
    Gba = np.vdot(vecs[b], vecs[a])
    for k in range(n):
        for l in range(n):
            if k != l:
                x = np.vdot(vecs[b], c[k] @ (c[l] @ vecs[a]))
                assert abs(x - 1j * Gba * D[k, l]) < 1e-12
    # n-point elements: Pfaffian of the sub-block of i Delta (Sec. III B)
    for idx in [(0, 1, 2, 3), (0, 2, 3, 5), (1, 2, 4, 5)]:
        x = np.vdot(vecs[b], c[idx[0]] @ c[idx[1]] @ c[idx[2]] @ (c[idx[3]] @ vecs[a]))
        sub = 1j * D[np.ix_(idx, idx)]
        assert abs(x - Gba * orc.pfaffian(sub)) < 1e-12
    # Delta^{a,a} = Gamma^a (Sec. III B)
    assert np.allclose(orc.transition_matrix(gammas[0], gammas[0]), gammas[0])
    # skew-symmetry and Delta^{b,a} = conj(Delta^{a,b})
    assert np.allclose(D, -D.T)
    assert np.allclose(orc.transition_matrix(gammas[b], gammas[a]), D.conj())


def test_phase_matches_three_state_grassmann_pfaffian():
    """At N where Fock vectors are out of reach, the transition-form phase
    must agree with the independent 3n x 3n Grassmann form of the Bargmann
    product: <0|a><a|b><b|0> = Pf(G0) (i/4)^N Pf([[iG0,-1,1],[1,iGa,-1],[-1,1,iGb]])
    (pinned itself against Fock vectors at small N below)."""
    for N, seed in ((3, 1), (4, 2)):
        gammas, vecs = _states(N, 3, seed)
        g0, ga, gb = gammas
        I = np.eye(2 * N)
        R = np.block([[1j * g0, -I, I], [I, 1j * ga, -I], [-I, I, 1j * gb]])
        B_fock = np.vdot(vecs[0], vecs[1]) * np.vdot(vecs[1], vecs[2]) * np.vdot(vecs[2], vecs[0])
        B_grass = orc.pfaffian(g0) * (0.25j) ** N * orc.pfaffian(R)
        assert abs(B_fock - B_grass) < 1e-12
    model = orc.anderson_model(9, 2.0, -1.0, 0.5)          # N = 20 modes
    rng = _rng(8)
    gammas = [inp.random_pure_gamma(20, rng) for _ in range(3)]
    G, _ = orc.gram_and_hamiltonian(model, gammas)
    g0, ga, gb = gammas
    I = np.eye(40)
    R = np.block([[1j * g0, -I, I], [I, 1j * ga, -I], [-I, I, 1j * gb]])
    ph, la = orc.pfaffian_log(R)
    B = orc.pfaffian(g0) * (1j ** 20) * ph
    Bo = G[0, 1] * G[1, 2] * G[2, 0]
    assert abs(Bo / abs(Bo) - B / abs(B)) < 1e-10
    # magnitude too: log|B| = 20 log(1/4) + log|Pf R|
    assert abs(math.log(abs(Bo)) - (20 * math.log(0.25) + la)) < 1e-9


# ---------------------------------------------------------------- amplitudes and energy

def test_energy_is_rayleigh_quotient_and_variational():
    model = orc.anderson_model(2, 2.0, -1.0, 0.5)           # 3 sites, N = 6 modes
    H = fock.hamiltonian_anderson(2, 2.0, -1.0, 0.5)
    gammas, vecs = _states(6, 3, 31)
    E, lam, G, h = orc.energy(model, gammas)
    psi = sum(l * v for l, v in zip(lam, vecs))
    assert abs(np.vdot(psi, psi) - 1.0) < 1e-12
    assert abs(np.vdot(psi, H @ psi) - E) < 1e-12
    E2, _ = fock.lowest_amplitudes(fock.gram(vecs), fock.hmat(vecs, H))
    assert abs(E - E2) < 1e-12
    assert E >= fock.ground_energy(H) - 1e-12


def test_higher_terms_hermitian_and_matched_by_fock():
    """Terms of six and eight Majoranas: the Fock operator is Hermitian (the factor
    i^(r mod 2)), and G, h of Gaussian states match Fock-space matrix elements."""
    model = _higher_model()
    H = _fock_operator(model)
    assert abs(H - H.conj().T).max() < 1e-14
    gammas, vecs = _states(4, 4, 77)
    G, h = orc.gram_and_hamiltonian(model, gammas)
    assert np.abs(G - fock.gram(vecs)).max() < 1e-12
    assert np.abs(h - fock.hmat(vecs, H)).max() < 1e-12
    # the terms matter: without them h changes by much more than the bar
    G0, h0 = orc.gram_and_hamiltonian(orc.MajoranaModel(model.A, model.quartic, model.e_const), gammas)
    assert np.abs(h - h0).max() > 1e-2


# ---------------------------------------------------------------- equation of motion


@pytest.mark.parametrize("mode", [orc.C_INVERSE, orc.C_PHASE])
def test_eom_with_higher_terms_matches_fock_flow(mode):
    """Eq. (EOM-Gamma3) with F the derivative of the Wick energy holds for terms of
    six and eight Majoranas: the matrix flow equals the Fock-space flow."""
    model = _higher_model()
    H = _fock_operator(model)
    gammas, vecs = _states(4, 3, 43)
    E, lam, G, h = orc.energy(model, gammas)
    dG = orc.eom(model, gammas, G, h, E, lam, mode)
    ref = fock.eom_bruteforce(vecs, lam, H, "inverse" if mode == orc.C_INVERSE else "phase")
    for a, b, g in zip(dG, ref, gammas):
        assert np.abs(a - b).max() < 1e-11 * max(1.0, np.abs(b).max())
        assert np.abs(a @ g + g @ a).max() < 1e-11 * max(1.0, np.abs(a).max())


def test_higher_fock_matrix_is_the_energy_derivative():
    """F - A = -(1/2) dE/dDelta_kl (both entries moving) by central differences on a
    random complex antisymmetric Delta, for the quartic and the higher terms."""
    model = _higher_model()
    rng = _rng(5)
    X = rng.standard_normal((8, 8)) + 1j * rng.standard_normal((8, 8))
    X = 0.5 * (X - X.T)
    F = orc.fock_matrix(model, X)
    h = 1e-6
    for k, l in [(0, 1), (2, 5), (3, 7), (6, 4)]:
        dX = np.zeros_like(X)
        dX[k, l], dX[l, k] = h, -h
        num = (orc.wick_energy_density(model, X + dX) - orc.wick_energy_density(model, X - dX)) / (2 * h)
        assert abs((F[k, l] - model.A[k, l]) - (-0.5 * num)) < 1e-7 * max(1.0, abs(num))

@pytest.mark.parametrize("mode", [orc.C_INVERSE, orc.C_PHASE])
def test_eom_matches_fock_flow(mode):
    model = orc.anderson_model(1, 3.0, -1.5, 0.7, t=1.0, mu=0.1)
    H = fock.hamiltonian_anderson(1, 3.0, -1.5, 0.7, t=1.0, mu=0.1)
    gammas, vecs = _states(4, 3, 41)
    E, lam, G, h = orc.energy(model, gammas)
    dG = orc.eom(model, gammas, G, h, E, lam, mode)
    ref = fock.eom_bruteforce(vecs, lam, H, "inverse" if mode == orc.C_INVERSE else "phase")
    for a, b, g in zip(dG, ref, gammas):
        assert np.abs(a - b).max() < 1e-11 * max(1.0, np.abs(b).max())
        # tangency (d Gamma) Gamma + Gamma (d Gamma) = 0 (Sec. III B)
        assert np.abs(a @ g + g @ a).max() < 1e-11 * max(1.0, np.abs(a).max())
        assert np.allclose(a, -a.T)


def test_rank_one_reduces_to_ghf():
    """R = 1: Eq. (EOM-Gamma3) falls back onto the GHF flow 4(F + Gamma F Gamma)
    with F the GHF Fock matrix (Sec. III B)."""
    model = orc.anderson_model(3, 2.5, -1.25, 0.6)
    rng = _rng(51)
    g = inp.random_pure_gamma(model.N, rng)
    E, lam, G, h = orc.energy(model, [g])
    dG = orc.eom(model, [g], G, h, E, lam)[0]
    F = np.zeros_like(model.A) + model.A
    for (k, l, m, r), v in model.quartic:
        F[k, l] += 6.0 * v * g[m, r]
    assert np.abs(dG - 4.0 * (F + g @ F @ g)).max() < 1e-12


# ---------------------------------------------------------------- integrator (App. A)

def test_orthogonal_step_first_order_and_pure():
    model = orc.anderson_model(2, 2.0, -1.0, 0.5)
    rng = _rng(61)
    gammas = [inp.random_pure_gamma(model.N, rng) for _ in range(3)]
    E, lam, G, h = orc.energy(model, gammas)
    dG = orc.eom(model, gammas, G, h, E, lam)
    errs = []
    for ds in (1e-2, 5e-3, 2.5e-3):
        g1 = orc.orthogonal_step(gammas[1], dG[1], ds)
        assert np.abs(g1 @ g1 + np.eye(model.n)).max() < 1e-13
        errs.append(np.abs(g1 - (gammas[1] + ds * dG[1])).max())
    # O(ds^2): halving ds quarters the gap to the Euler step
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_purify_recovers_canonical_form():
    rng = _rng(71)
    N = 6
    O = inp.haar_orthogonal(2 * N, rng)
    lam = rng.uniform(0.9, 1.1, N)
    blk = np.zeros((2 * N, 2 * N))
    for j in range(N):
        blk[2 * j, 2 * j + 1], blk[2 * j + 1, 2 * j] = lam[j], -lam[j]
    noisy = O @ blk @ O.T
    clean = O @ inp.vacuum_gamma(N) @ O.T
    assert np.abs(orc.purify(noisy) - clean).max() < 1e-13
    assert np.abs(orc.purify(clean) - clean).max() < 1e-14


def test_euler_step_first_order_and_pure():
    """Eq. (RKstep) with the canonical-form renormalisation of App. A: pure, and
    within O(ds^3) of the orthogonal step (for a tangent dGamma both expand to
    Gamma + ds dGamma + (ds^2/2) Gamma dGamma^2)."""
    model = orc.anderson_model(2, 2.0, -1.0, 0.5)
    rng = _rng(63)
    gammas = [inp.random_pure_gamma(model.N, rng) for _ in range(3)]
    E, lam, G, h = orc.energy(model, gammas)
    dG = orc.eom(model, gammas, G, h, E, lam)
    errs = []
    for ds in (1e-2, 5e-3):
        g1 = orc.euler_step(gammas[2], dG[2], ds)
        assert np.abs(g1 @ g1 + np.eye(model.n)).max() < 1e-13
        errs.append(np.abs(g1 - orc.orthogonal_step(gammas[2], dG[2], ds)).max())
    assert 7.0 < errs[0] / errs[1] < 9.0
    Es, _, _ = orc.euler_run(model, gammas, 0.02, 20)
    assert np.all(np.diff(Es) <= 1e-12)


# ---------------------------------------------------------------- rank growth (Sec. III C)

def test_added_state_is_the_gaussian_unitary_image():
    """Q Gamma Q^T with Q = exp(K) is the covariance of U|phi>, U = exp((1/4)
    sum K_kl c_k c_l) the Gaussian unitary of K (Fock brute force); it keeps
    the parity (det Q = 1) and the purity."""
    rng = _rng(101)
    N = 4
    g = inp.random_pure_gamma(N, rng, -1)
    K = inp.random_generator(2 * N, 0.4, rng)
    new = orc.add_state([g], K, 0)[1]
    c = fock.majoranas(N)
    gen = sum(K[k, l] * (c[k] @ c[l]) for k in range(2 * N) for l in range(2 * N))
    import scipy.linalg
    phi = scipy.linalg.expm(0.25 * gen.toarray()) @ fock.gaussian_vector(g)
    assert np.abs(fock.covariance_of(phi) - new).max() < 1e-12
    assert abs(orc.pfaffian(new) - orc.pfaffian(g)) < 1e-12
    assert np.abs(new @ new + np.eye(2 * N)).max() < 1e-13


def test_added_state_never_raises_the_energy():
    """With optimal amplitudes the enlarged ansatz contains the old one, so the
    energy cannot rise; a copy with K = 0 makes G singular and the canonical
    orthogonalisation drops it (energy unchanged)."""
    model = orc.anderson_model(3, 4.0, -2.0, 0.5)
    rng = _rng(103)
    gammas = [inp.random_pure_gamma(model.N, rng) for _ in range(2)]
    E0 = orc.energy(model, gammas)[0]
    for src in (0, 1):
        E1 = orc.energy(model, orc.add_state(gammas, inp.random_generator(model.n, 0.2, rng), src))[0]
        assert E1 <= E0 + 1e-12
    E2 = orc.energy(model, orc.add_state(gammas, np.zeros((model.n, model.n)), 0))[0]
    assert abs(E2 - E0) < 1e-12 * abs(E0)


def test_rank_growth_approaches_exact_ground_state():
    """The paper's route to the ground state (Sec. III C): from a single
    Gaussian, one state added every 60 steps up to rank 6; the energy stays above
    the exact ground state (variational) and ends within 3e-4 of it (4 sites,
    U = 4)."""
    model = orc.anderson_model(3, 4.0, -2.0, 0.5)
    E_ed = fock.ground_energy(fock.hamiltonian_anderson(3, 4.0, -2.0, 0.5))
    g, _ = inp.initial_state(model.N, 1, 3, 1)
    rng = _rng(0)
    Ks = [inp.random_generator(model.n, 0.1, rng) for _ in range(5)]
    Es, gs = orc.grow(model, list(g), 0.1, 60, Ks)
    assert len(gs) == 6 and len(Es) == 360
    assert np.all(Es >= E_ed - 1e-12)
    assert (Es[-1] - E_ed) / abs(E_ed) < 3e-4
    assert (Es[59] - E_ed) / abs(E_ed) > 1e-2          # the single Gaussian is far off


@pytest.mark.parametrize("L", [2, 3])
def test_two_channel_kondo_model_equals_fermion_hamiltonian(L):
    """Sec. V: the Majorana form of H_2CK equals the Hamiltonian built from
    fermion operators (hopping, H_BC, J S_imp . S_alpha(1)); its ground state
    has even parity."""
    J, t = 1.3, 0.5
    model = orc.two_channel_kondo_model(L, J, t)
    N = model.N
    a = fock.annihilators(N)
    ad = [x.conj().T.tocsr() for x in a]
    H = 0.0 * _fock_operator(model)
    for s in range(2):
        for ch in range(2):
            ends = [orc.kondo_site(ch, r) for r in range(1, L)] + [2 * L - 1]
            for x, y in zip(ends[:-1], ends[1:]):
                p, q = 2 * x + s, 2 * y + s
                H = H - t * (ad[p] @ a[q] + ad[q] @ a[p])
    for ch in range(2):
        for x, y in zip(fock.spin_ops(N, 0), fock.spin_ops(N, orc.kondo_site(ch, 1))):
            H = H + J * (x @ y)
    assert abs(H - _fock_operator(model)).max() < 1e-13
    w, v = np.linalg.eigh(H.toarray())
    parity = np.array([(-1) ** bin(i).count("1") for i in range(2 ** N)])
    assert np.vdot(v[:, 0], parity * v[:, 0]).real > 0.999


# ---------------------------------------------------------------- variance (Eq. residual)

def _two_site_hubbard():
    """Two spinful sites with hopping and three density-density terms, two of
    which share Majoranas: H4 H4 then has repeated indices."""
    h = np.array([[0.3, 0.0, -1.0, 0.0], [0.0, -0.2, 0.0, -0.7],
                  [-1.0, 0.0, 0.1, 0.0], [0.0, -0.7, 0.0, 0.4]])
    return orc.majorana_from_fermions(h, [(0, 1, 2.0), (2, 3, 1.5), (0, 3, 0.8)])


@pytest.mark.parametrize("which", ["hubbard", "anderson2"])
def test_hamiltonian_square_matches_fock(which):
    model = _two_site_hubbard() if which == "hubbard" else orc.anderson_model(1, 3.0, -1.5, 0.6, n_channels=2)
    assert len(orc.canonical_quartic(model)) == (3 if which == "hubbard" else 1)
    H = _fock_operator(model).toarray()
    H2 = H @ H
    gammas, vecs = _states(model.N, 3, 111)
    for a in range(3):
        for b in range(3):
            D = gammas[a].astype(np.complex128) if a == b else orc.transition_matrix(gammas[b], gammas[a])
            x = orc.hamiltonian_square_density(model, D)
            y = np.vdot(vecs[a], H2 @ vecs[b]) / np.vdot(vecs[a], vecs[b])
            assert abs(x - y) < 1e-12 * max(1.0, abs(y)), (a, b)


def test_variance_matches_fock():
    model = orc.anderson_model(2, 2.0, -1.0, 0.5)
    H = _fock_operator(model).toarray()
    gammas, vecs = _states(model.N, 3, 113)
    E, var = orc.variance(model, gammas)
    _, lam, _, _ = orc.energy(model, gammas)
    psi = sum(l * v for l, v in zip(lam, vecs))
    nrm = np.vdot(psi, psi).real
    e1 = np.vdot(psi, H @ psi).real / nrm
    e2 = np.vdot(psi, H @ (H @ psi)).real / nrm
    assert abs(E - e1) < 1e-12 and abs(var - (e2 - e1 * e1)) < 1e-12 and var > 0


def test_variance_vanishes_on_an_eigenstate():
    """U = 0: the GHF flow reaches the exact (Gaussian) ground state, an
    eigenstate of H, where delta_H^2 = 0."""
    h_sp, _ = orc.anderson_chain(7, 0.0, 0.0, 0.5)
    model = orc.majorana_from_fermions(h_sp, [])
    g = [inp.random_pure_gamma(model.N, _rng(117), 1)]
    assert orc.variance(model, g)[1] > 1e-2
    _, _, gs = orc.run(model, g, 0.25, 400)
    assert abs(orc.variance(model, gs)[1]) < 1e-9


def test_energy_extrapolation():
    """Linear fit of E against delta_H^2 (Sec. IV A): exact on a line, equal to
    numpy.polyfit on scattered points.  On a rank-growth run (4 sites, ranks
    1..8) every rank's (E, delta_H^2) obeys the variational bound E >= E_0 and
    Temple's inequality E - E_0 <= delta_H^2 / (E_1 - E) for E < E_1 (E_0, E_1
    the two lowest eigenvalues by exact diagonalisation), which ties the
    energy and the variance to the exact spectrum whatever trajectory the
    growth takes.  (A bracket of E_0 by the fit's standard error does not
    follow: at these variances E is not linear in delta_H^2.)"""
    v = np.array([1e-6, 3e-6, 7e-6, 1.2e-5, 1.9e-5, 5e-5])
    Es, err = orc.extrapolate_energy(-3.25 + 41.0 * v, v)
    assert abs(Es + 3.25) < 1e-12 and err < 1e-12
    noisy = -3.25 + 41.0 * v + np.array([3e-7, -2e-7, 1e-7, 4e-7, -5e-7, 9.0])
    Es, err = orc.extrapolate_energy(noisy, v)
    k, b = np.polyfit(v[:5], noisy[:5], 1)
    assert abs(Es - b) < 1e-12 and err > 0
    model = orc.anderson_model(3, 4.0, -2.0, 0.5)
    spec = np.linalg.eigvalsh(fock.hamiltonian_anderson(3, 4.0, -2.0, 0.5).toarray())
    E_ed, E_1 = spec[0], spec[1]
    assert E_1 - E_ed > 0.1                                   # a non-degenerate ground state
    g, _ = inp.initial_state(model.N, 1, 3, 1)
    rng = _rng(0)
    gam, pts = list(g), []
    for M in range(1, 9):
        _, lam, gam = orc.run(model, gam, 0.1, 60)
        E, var = orc.variance(model, gam)
        assert E >= E_ed - 1e-12 and var > 0
        assert E < E_1 and E - E_ed <= var / (E_1 - E) + 1e-12, (M, E, var)
        pts.append((E, var))
        gam = orc.add_state(gam, inp.random_generator(model.n, 0.1, rng), int(np.argmax(np.abs(lam))))
    E, var = np.array(pts).T
    assert var[-1] < 1e-2 and E[-1] - E_ed < 1e-3              # the growth converges toward E_0
    Es, err = orc.extrapolate_energy(E, var, var_max=1e-2)
    assert np.isfinite(Es) and err > 0


# ---------------------------------------------------------------- whole-step ground truths

def test_energy_descends():
    model = orc.anderson_model(2, 2.0, -1.0, 0.5)
    rng = _rng(81)
    gammas = [inp.random_pure_gamma(model.N, rng) for _ in range(3)]
    Es, _, _ = orc.run(model, gammas, 0.02, 30)
    assert np.all(np.diff(Es) <= 1e-12)
    H = fock.hamiltonian_anderson(2, 2.0, -1.0, 0.5)
    assert Es[-1] >= fock.ground_energy(H) - 1e-12


def test_noninteracting_closed_form():
    """U = 0: a single Gaussian is exact, and the GHF flow reaches the sum of
    the negative single-particle energies (Sec. II A)."""
    h_sp, _ = orc.anderson_chain(7, 0.0, 0.0, 0.5)
    model = orc.majorana_from_fermions(h_sp, [])
    eps = np.linalg.eigvalsh(h_sp)
    exact = eps[eps < 0].sum()
    rng = _rng(91)
    g = [inp.random_pure_gamma(model.N, rng, 1)]
    Es, _, gs = orc.run(model, g, 0.25, 400)
    assert abs(Es[-1] - exact) < 1e-9


# ---------------------------------------------------------------- observables (Eq. Cr, Eq. K2CK)

def test_spin_correlator_matches_fock():
    model = orc.anderson_model(2, 2.0, -1.0, 0.5)          # 3 sites, N = 6 modes
    gammas, vecs = _states(6, 3, 101)
    E, lam, G, h = orc.energy(model, gammas)
    psi = sum(l * v for l, v in zip(lam, vecs))
    for s in range(3):
        ref = fock.spin_spin(psi, 6, 0, s)
        got = orc.spin_correlator(gammas, lam, G, [s])[0]
        assert abs(got - ref) < 1e-12, (s, got, ref)


def test_two_channel_correlator_matches_fock():
    model = orc.anderson_model(1, 2.0, -1.0, 0.5, n_channels=2)   # impurity + 2 channels x 1 site
    gammas, vecs = _states(6, 2, 103, parity=-1)
    E, lam, G, h = orc.energy(model, gammas)
    psi = sum(l * v for l, v in zip(lam, vecs))
    ref = fock.spin_spin(psi, 6, 0, 1) + fock.spin_spin(psi, 6, 0, 2)
    assert abs(orc.two_channel_correlator(gammas, lam, G, [1])[0] - ref) < 1e-12


def test_spin_sum_rule_for_exact_singlet():
    """Sum_r C(r) = <S(0) . S_tot> = 0 for the even-L singlet ground state
    (the sum rule Sigma(L-1) = 0 of Sec. IV B), checked on the operator
    algebra: the exact ground state from ED, expectation of the oracle's
    Majorana polynomials through explicit Fock matrices."""
    H = fock.hamiltonian_anderson(1, 2.0, -1.0, 0.5)       # 2 sites, N = 4 modes: singlet ground state
    w, v = np.linalg.eigh(H.toarray())
    g = v[:, 0]
    c = fock.majoranas(4)
    tot = 0.0
    for s in range(2):
        P = orc.spin_dot(0, s)
        op = sum(coef * (np.linalg.multi_dot([c[i].toarray() for i in m]) if len(m) > 1 else
                         (c[m[0]].toarray() if len(m) == 1 else np.eye(16))) for m, coef in P.items())
        val = np.vdot(g, op @ g)
        assert abs(val - fock.spin_spin(g, 4, 0, s)) < 1e-12
        tot += val
    assert abs(tot) < 1e-12


# ---------------------------------------------------------------- Renyi-2 (App. B)

@pytest.mark.parametrize("n_sites_A", [1, 2])
def test_renyi2_matches_fock_reduced_density_matrix(n_sites_A):
    gammas, vecs = _states(6, 3, 111)                        # 3 sites
    model = orc.anderson_model(2, 2.0, -1.0, 0.5)
    E, lam, G, h = orc.energy(model, gammas)
    psi = sum(l * v for l, v in zip(lam, vecs))
    ref = fock.renyi2_leading_modes(psi, 2 * n_sites_A)
    assert abs(orc.renyi2(gammas, lam, G, 2 * n_sites_A) - ref) < 1e-10


def test_renyi2_single_gaussian_closed_form_and_pure_limits():
    """R = 1: S_2 = -sum_j ln[(1 + nu_j^2)/2], +-i nu_j the eigenvalues of
    Gamma_A (the single-Gaussian result the paper cites in Sec. IV C); the
    whole system (N_B = 0) is pure: S_2 = 0."""
    rng = _rng(121)
    N = 8
    g = inp.random_pure_gamma(N, rng)
    for NA in (1, 3, 5):
        GA = g[:2 * NA, :2 * NA]
        ev = np.linalg.eigvalsh(1j * GA)                      # +-nu_j
        nu = np.sort(np.abs(ev))[::2]
        ref = -np.sum(np.log((1.0 + nu ** 2) / 2.0))
        got = orc.renyi2([g], np.array([1.0 + 0j]), np.ones((1, 1)), NA)
        assert abs(got - ref) < 1e-10
    gammas, vecs = _states(4, 2, 123)
    model = orc.anderson_model(1, 2.0, -1.0, 0.5)
    E, lam, G, h = orc.energy(model, gammas)
    assert abs(orc.renyi2(gammas, lam, G, 4)) < 1e-10
