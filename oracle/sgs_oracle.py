"""Plain FP64 CPU oracle for one imaginary-time step of the superposition-of-
Gaussian-states (SGS) variational method (Boutin & Bauer, arXiv:2105.01088).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
reference against which the CUDA path is checked.  Only the test-suite, the
package smoke check and the CPU-baseline leg of the benchmark may import it;
the product path never does, and the CUDA path shares no code with it.

Everything is numpy float64 / complex128.  Library primitives used as single
steps: ``numpy.linalg.slogdet`` (log|det|), ``numpy.linalg.solve`` (a linear
solve), ``numpy.linalg.eigh`` (Hermitian eigen-decomposition),
``scipy.linalg.expm`` (matrix exponential).  The Pfaffian is written out here
(Parlett-Reid elimination with pivoting), as the paper's PFAPACK is not used.

Conventions (the paper fixes none of these; each is a stated reading):
  * Majoranas c_{2m}, c_{2m+1} of fermion mode m (0-based) are
    a_m + a_m^dag and -i(a_m - a_m^dag); the vacuum then has Gamma = J,
    J = (+)_m [[0, 1], [-1, 0]], and the parity of a Gaussian state is Pf(Gamma).
  * Mode order is site-major, spin-minor: mode 2s+sigma, impurity site s=0.
  * The gauge reference state of Sec. II B is the first ansatz state, phi_0.
  * Eq. (EOM-Gamma3) is used with lambda-tilde_mu conjugated (as in
    Eq. (EOM-Gamma2)), and with its last term summed through h lambda = E G
    lambda (Eq. eigLambda), so the bracket ends in -(h_mu,beta - E G_mu,beta)
    Delta^{beta,mu}.
  * The orthogonal step of App. A (Eq. ExpStep) uses
    R = exp{(ds/4)[Gamma, dGamma]}, which agrees with the Euler step
    Gamma + ds dGamma (Eq. RKstep) to first order in ds.

Parity pins (tests/test_oracle_pins.py): every function here is checked
against explicit Fock-space vectors, exact diagonalisation, the U=0 closed
form or a paper-stated identity; none is "parity unpinned".
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.linalg

# ---------------------------------------------------------------------------
# Model: fermion Hamiltonian -> Majorana form (Sec. II A; Sec. IV Eqs. for
# H_0, H_I; Sec. V two-channel geometry)
# ---------------------------------------------------------------------------


class MajoranaModel:
    """H = e_const + i sum_kl A_kl c_k c_l + sum_klpq U_klpq c_k c_l c_p c_q
         + sum_j v_j i^(r_j mod 2) c_{s_j1} ... c_{s_j(2 r_j)}.

    ``A`` is the real skew 2N x 2N matrix of Sec. II A.  The quartic tensor is
    kept as its non-zero antisymmetrised entries: ``quartic`` is a list of
    ((k, l, p, q), value) with the value of U_klpq for every ordering of each
    monomial's four distinct indices (Sec. II A: U is skew under exchange of
    neighbouring indices, hence fully antisymmetric).  ``higher`` holds
    interaction terms of more than four Majoranas (Sec. II A allows them; Sec.
    III C estimates their cost), as (indices, v): 2r distinct indices, r >= 3,
    and a real v; the factor i^(r mod 2) makes the term Hermitian, since the
    product of 2r distinct Majoranas is Hermitian for even r and anti-Hermitian
    for odd r.
    """

    def __init__(self, A, quartic, e_const, higher=()):
        self.A = np.asarray(A, dtype=np.float64)
        self.quartic = list(quartic)
        self.higher = [(tuple(int(x) for x in idx), float(v)) for idx, v in higher]
        for idx, _ in self.higher:
            assert len(idx) % 2 == 0 and len(idx) >= 6 and len(set(idx)) == len(idx)
        self.e_const = float(e_const)
        self.n = self.A.shape[0]
        self.N = self.n // 2


def _perm_sign(p):
    s = 1
    p = list(p)
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if p[i] > p[j]:
                s = -s
    return s


def antisymmetrise_monomials(monomials):
    """Turn monomials v * c_k c_l c_p c_q (distinct k,l,p,q) into the fully
    antisymmetric U of Sec. II A: U_{pi(klpq)} = sgn(pi) v / 24, so that
    sum over all orderings reproduces v c_k c_l c_p c_q."""
    out = {}
    for idx, v in monomials:
        assert len(set(idx)) == 4, "quartic monomial needs four distinct Majoranas"
        for perm in itertools.permutations(range(4)):
            key = tuple(idx[i] for i in perm)
            out[key] = out.get(key, 0.0) + _perm_sign(perm) * v / 24.0
    return [(k, v) for k, v in out.items() if v != 0.0]


def majorana_from_fermions(h_sp, hubbard):
    """Quadratic fermion part sum_ij h_ij a_i^dag a_j (h real symmetric) and
    Hubbard terms U n_a n_b (list of (a, b, U), a != b) -> MajoranaModel.

    With a_m = (c_{2m} + i c_{2m+1})/2:
      sum_ij h_ij a_i^dag a_j = tr(h)/2 + (i/2) sum_ij h_ij c_{2i} c_{2j+1},
    i.e. A_{2i,2j+1} = h_ij / 4 = -A_{2j+1,2i}.  With n_m = (1 + i c_{2m}
    c_{2m+1})/2, U n_a n_b = U/4 + (U/4)(i c c)_a + (U/4)(i c c)_b
    - (U/4) c_{2a} c_{2a+1} c_{2b} c_{2b+1}.
    """
    h_sp = np.asarray(h_sp, dtype=np.float64)
    nm = h_sp.shape[0]
    n = 2 * nm
    A = np.zeros((n, n))
    e_const = 0.5 * np.trace(h_sp)
    for i in range(nm):
        for j in range(nm):
            if h_sp[i, j] != 0.0:
                A[2 * i, 2 * j + 1] += h_sp[i, j] / 4.0
                A[2 * j + 1, 2 * i] -= h_sp[i, j] / 4.0
    monomials = []
    for a, b, U in hubbard:
        e_const += U / 4.0
        for m in (a, b):
            A[2 * m, 2 * m + 1] += U / 8.0
            A[2 * m + 1, 2 * m] -= U / 8.0
        monomials.append(((2 * a, 2 * a + 1, 2 * b, 2 * b + 1), -U / 4.0))
    return MajoranaModel(A, antisymmetrise_monomials(monomials), e_const)


def anderson_chain(n_bath, U, eps_d, V, t=1.0, mu=0.0, n_channels=1):
    """Single-impurity Anderson model of Sec. IV (H_0 + H_I), generalised to
    ``n_channels`` independent open bath chains of ``n_bath`` sites each,
    every chain's first site hybridised with the impurity by V (= t').

    Site order: impurity s=0, then the chains interleaved by channel
    (channel c, chain site r = 1..n_bath -> s = 1 + (r-1)*n_channels + c),
    so "impurity + first k chain sites of every channel" is a leading block.
    Mode 2s + sigma.  Returns (h_sp, hubbard) for majorana_from_fermions.
    """
    n_sites = 1 + n_channels * n_bath
    nm = 2 * n_sites
    h = np.zeros((nm, nm))

    def site(c, r):
        return 1 + (r - 1) * n_channels + c

    for sigma in range(2):
        h[sigma, sigma] = eps_d
        for c in range(n_channels):
            a, b = 0, site(c, 1)
            h[2 * a + sigma, 2 * b + sigma] = h[2 * b + sigma, 2 * a + sigma] = -V
            for r in range(1, n_bath + 1):
                s = site(c, r)
                h[2 * s + sigma, 2 * s + sigma] = -mu
                if r >= 2:
                    p = site(c, r - 1)
                    h[2 * p + sigma, 2 * s + sigma] = h[2 * s + sigma, 2 * p + sigma] = -t
    return h, [(0, 1, U)]


def anderson_model(n_bath, U, eps_d, V, t=1.0, mu=0.0, n_channels=1):
    return majorana_from_fermions(*anderson_chain(n_bath, U, eps_d, V, t, mu, n_channels))


def kondo_site(ch, r):
    """Site of channel ch (0, 1) at distance r (1 .. L-1) in the two-channel
    Kondo lattice; the impurity is site 0 and the boundary site 2L - 1."""
    return 1 + 2 * (r - 1) + ch


def two_channel_kondo_model(L, J, t=0.5):
    """H_2CK of Sec. V: two channels of L - 1 sites with hopping -t, the
    boundary site joining their far ends (H_BC), and H_J = J sum_alpha S_imp .
    S_alpha(1) with a fermionic impurity that has no quadratic term (2L sites in
    all).  The quadratic part goes through majorana_from_fermions; H_J is
    expanded into Majorana monomials by the polynomial algebra below."""
    n_sites = 2 * L
    nm = 2 * n_sites
    h = np.zeros((nm, nm))
    bc = n_sites - 1
    for s in range(2):
        for ch in range(2):
            for r in range(2, L):
                p, q = 2 * kondo_site(ch, r - 1) + s, 2 * kondo_site(ch, r) + s
                h[p, q] = h[q, p] = -t
            p, q = 2 * kondo_site(ch, L - 1) + s, 2 * bc + s
            h[p, q] = h[q, p] = -t
    base = majorana_from_fermions(h, [])
    monomials = []
    for ch in range(2):
        for mono, coef in spin_dot(0, kondo_site(ch, 1)).items():
            assert len(mono) == 4 and abs(np.imag(coef)) < 1e-15, (mono, coef)
            monomials.append((mono, J * float(np.real(coef))))
    return MajoranaModel(base.A, antisymmetrise_monomials(monomials), base.e_const)


# ---------------------------------------------------------------------------
# Pfaffian (the paper computes Pfaffians with PFAPACK; this is a plain
# Parlett-Reid elimination with partial pivoting)
# ---------------------------------------------------------------------------


def pfaffian_log(A):
    """Return (phase, log|Pf A|) of a real or complex skew matrix A, with
    Pf A = phase * exp(log|Pf A|).  phase is +-1 for real A.  A zero pivot
    returns (0, -inf)."""
    A = np.array(A, dtype=np.complex128 if np.iscomplexobj(A) else np.float64)
    n = A.shape[0]
    if n % 2:
        return 0.0, -math.inf
    phase = 1.0 + 0.0j if np.iscomplexobj(A) else 1.0
    logabs = 0.0
    for k in range(0, n - 1, 2):
        # pivot: largest entry of column k below the diagonal
        p = k + 1 + int(np.argmax(np.abs(A[k + 1:, k])))
        if p != k + 1:
            A[[k + 1, p], :] = A[[p, k + 1], :]
            A[:, [k + 1, p]] = A[:, [p, k + 1]]
            phase = -phase
        piv = A[k, k + 1]
        if piv == 0:
            return 0.0, -math.inf
        logabs += math.log(abs(piv))
        phase = phase * (piv / abs(piv))
        if k + 2 < n:
            tau = A[k, k + 2:] / piv
            u = A[k + 2:, k + 1].copy()
            A[k + 2:, k + 2:] += np.outer(tau, u) - np.outer(u, tau)
    return phase, logabs


def pfaffian(A):
    ph, la = pfaffian_log(A)
    return ph * math.exp(la) if la > -math.inf else 0.0 * ph


# ---------------------------------------------------------------------------
# Pair quantities (Sec. II B-C, Sec. III B)
# ---------------------------------------------------------------------------


def log_overlap_magnitude(Ga, Gb):
    """log |<phi_a|phi_b>| from |<phi_a|phi_b>|^2 = 2^-N |Pf(Ga + Gb)|
    (overlap magnitude of Gaussian states, Sec. II B, following the paper's
    Ref. [Bravyi2017]); |Pf S| = |det S|^(1/2)."""
    N = Ga.shape[0] // 2
    sign, logdet = np.linalg.slogdet(Ga + Gb)
    if sign == 0:
        return -math.inf
    return 0.5 * (-N * math.log(2.0) + 0.5 * logdet)


def transition_matrix(Ga, Gb):
    """Delta^{a,b} = [i(Ga - Gb) - 2](Ga + Gb)^{-1}  (Eq. def-delta-matrix),
    so that <phi_b| c_k c_l |phi_a> = i G_{b,a} Delta^{a,b}_kl for k != l."""
    n = Ga.shape[0]
    S = Ga + Gb
    rhs = 1j * (Ga - Gb) - 2.0 * np.eye(n)
    # X S = rhs  <=>  S^T X^T = rhs^T
    return np.linalg.solve(S.T, rhs.T).T


def _higher_phase(r):
    """i^(r mod 2) (the term's factor) times i^r (the Pfaffian of i Delta): a sign."""
    return (-1.0) ** ((r + r % 2) // 2)


def wick_energy_density(model, Dlt):
    """<phi_b|H|phi_a> / <phi_b|phi_a> for the transition matrix Delta^{a,b}:
    e_const + Tr(A Delta) - 3 sum_klpq U_klpq Delta_kl Delta_pq, plus for each
    term of 2r > 4 Majoranas v i^(r mod 2) Pf(i Delta_S) = v (-1)^((r + r mod 2)/2)
    Pf(Delta_S), Delta_S the sub-block on the term's indices in its order.
    (Generalised Wick theorem of Sec. III B: two-point elements i Delta_kl, an
    element of n distinct Majoranas the Pfaffian of the n x n sub-block of
    i Delta.)"""
    e = model.e_const + np.sum(model.A * Dlt.T)
    q = 0.0
    for (k, l, p, r), v in model.quartic:
        q += v * Dlt[k, l] * Dlt[p, r]
    e = e - 3.0 * q
    for idx, v in model.higher:
        e = e + v * _higher_phase(len(idx) // 2) * pfaffian(Dlt[np.ix_(idx, idx)])
    return e


def fock_matrix(model, Dlt):
    """Generalised Fock matrix F^{a,b}_kl = A_kl + 6 sum_mn U_klmn Delta^{a,b}_mn
    (Sec. III B): F_kl = A_kl - (1/2) dE/dDelta_kl, the derivative of the Wick
    energy with Delta_kl and Delta_lk = -Delta_kl moving together.  For a term of
    2r > 4 Majoranas on positions a < b of its index list S, dPf(Delta_S)/dDelta_ab
    = (-1)^(a + b + 1) Pf(Delta_S without rows and columns a, b)."""
    F = model.A.astype(np.complex128 if np.iscomplexobj(Dlt) else np.float64).copy()
    for (k, l, m, r), v in model.quartic:
        F[k, l] += 6.0 * v * Dlt[m, r]
    if model.higher:
        F = F.astype(np.complex128) if np.iscomplexobj(Dlt) else F
    for idx, v in model.higher:
        c = v * _higher_phase(len(idx) // 2)
        sub = Dlt[np.ix_(idx, idx)]
        m = len(idx)
        for a in range(m):
            for b in range(a + 1, m):
                rest = [x for x in range(m) if x != a and x != b]
                d = (-1.0) ** (a + b + 1) * pfaffian(sub[np.ix_(rest, rest)])
                F[idx[a], idx[b]] += -0.5 * c * d
                F[idx[b], idx[a]] -= -0.5 * c * d
    return F


def gram_and_hamiltonian(model, gammas):
    """Gram matrix G_ab = <phi_a|phi_b> and h_ab = <phi_a|H|phi_b> (Sec. II C,
    Eq. eigLambda) in the gauge of Sec. II B with reference phi_0 = the first
    state: <phi_0|phi_mu> real and positive.

    Magnitude: |G_ab| from the Pfaffian of Ga + Gb.  Phase: the Bargmann
    product <phi_0|phi_a><phi_a|phi_b><phi_b|phi_0> equals
    |G_ab|^2 2^-N Pf(G0) Pf(G0 + Delta^{a,b}) (the trace of the reference
    projector against the transition operator |a><b|/<b|a>, whose two-point
    function is Delta^{a,b}); with <phi_0|phi_a>, <phi_b|phi_0> > 0 its phase
    is the phase of G_ab.
    """
    M = len(gammas)
    G = np.zeros((M, M), dtype=np.complex128)
    h = np.zeros((M, M), dtype=np.complex128)
    for a in range(M):
        G[a, a] = 1.0
        h[a, a] = wick_energy_density(model, gammas[a])
        for b in range(a + 1, M):
            G[a, b], h[b, a] = pair_elements(model, gammas, a, b)
            G[b, a] = np.conj(G[a, b])
            h[a, b] = np.conj(h[b, a])
    return G, h


def pair_elements(model, gammas, a, b):
    """(G_ab, h_ba) of one pair a < b in the gauge of the first state: the
    magnitude from Pf(Ga + Gb), the phase from the Bargmann product with the
    reference state (gram_and_hamiltonian), h_ba = G_ba * Wick(Delta^{a,b})."""
    Dab = transition_matrix(gammas[a], gammas[b])
    mag = math.exp(log_overlap_magnitude(gammas[a], gammas[b]))
    if a == 0:
        g = mag + 0.0j
    else:
        pf0, _ = pfaffian_log(gammas[0])
        ph, _ = pfaffian_log(gammas[0] + Dab)
        ph = ph * pf0
        g = mag * ph / abs(ph)
    # h_ba = <phi_b|H|phi_a> = G_ba * (Wick with Delta^{a,b})
    return g, np.conj(g) * wick_energy_density(model, Dab)


# ---------------------------------------------------------------------------
# Amplitudes (Eq. eigLambda)
# ---------------------------------------------------------------------------


def solve_amplitudes(G, h, rel_cut=1e-12):
    """Lowest solution of h lambda = E G lambda by canonical orthogonalisation:
    diagonalise G, keep eigenvalues above rel_cut * max, solve the ordinary
    Hermitian problem in that basis.  lambda is normalised to lambda^dag G
    lambda = 1 and its global phase set so the largest |lambda_mu| is real
    and positive.  Returns (E, lambda)."""
    w, U = np.linalg.eigh(G)
    keep = w > rel_cut * w.max()
    X = U[:, keep] / np.sqrt(w[keep])
    Hp = X.conj().T @ h @ X
    Hp = 0.5 * (Hp + Hp.conj().T)
    e, V = np.linalg.eigh(Hp)
    lam = X @ V[:, 0]
    lam = lam / math.sqrt(np.real(lam.conj() @ G @ lam))
    j = int(np.argmax(np.abs(lam)))
    lam = lam * (abs(lam[j]) / lam[j])
    return float(e[0]), lam


# ---------------------------------------------------------------------------
# Equation of motion (Sec. III A-B)
# ---------------------------------------------------------------------------

C_INVERSE = 0      # c_mu = [lambda_mu lambda-tilde_mu^*]^{-1}      (Sec. III A)
C_PHASE = 1        # c_mu = lambda-tilde_mu lambda_mu^* / |...|       (Sec. III A)


def coupling_constants(G, lam, mode=C_INVERSE, tiny=1e-300):
    """lambda-tilde = G lambda and the decoupling constants c_mu of Sec. III A.
    A state whose |lambda_mu lambda-tilde_mu| is below ``tiny`` gets c_mu = 0
    (its flow is frozen; the paper is silent on this case)."""
    lt = G @ lam
    c = np.zeros(len(lam), dtype=np.complex128)
    for m in range(len(lam)):
        z = lam[m] * np.conj(lt[m])
        if abs(z) < tiny:
            continue
        c[m] = 1.0 / z if mode == C_INVERSE else np.conj(z) / abs(z)
    return lt, c


def eom_term(model, gammas, G, h, E, lam, mu, beta):
    """The beta term of the sum of Eq. (EOM-Gamma3) for receiver mu,
    lambda_beta [ 2i G_mu,beta [D, F] + 2 G_mu,beta (D F D + F) - (h_mu,beta - E G_mu,beta) D ],
    with D = Delta^{beta,mu}, F = F^{beta,mu} and Delta^{mu,mu} = Gamma^mu (Sec. III B)."""
    D = gammas[mu].astype(np.complex128) if beta == mu else transition_matrix(gammas[beta], gammas[mu])
    F = fock_matrix(model, D)
    term = (2j * G[mu, beta] * (D @ F - F @ D)
            + 2.0 * G[mu, beta] * (D @ F @ D + F)
            - (h[mu, beta] - E * G[mu, beta]) * D)
    return lam[beta] * term


def eom(model, gammas, G, h, E, lam, mode=C_INVERSE, mus=None, betas=None):
    """d Gamma^mu / ds of Eq. (EOM-Gamma3), for every state mu:

    2 Re{ lt_mu^* c_mu sum_beta lambda_beta [ 2i G_mu,beta [D, F]
          + 2 G_mu,beta (D F D + F) - (h_mu,beta - E G_mu,beta) D ] }

    with D = Delta^{beta,mu}, F = F^{beta,mu}; "+ c.c." of the paper is
    X + X^* = 2 Re X.  Delta^{mu,mu} = Gamma^mu (Sec. III B).  ``mus``: the
    states to evaluate (default all).  ``betas(mu)``: the terms of the sum to
    take (default all beta); the expression is linear in them, so sums over a
    partition of the beta add up to the whole.
    """
    M = len(gammas)
    lt, c = coupling_constants(G, lam, mode)
    out = []
    for mu in (range(M) if mus is None else mus):
        acc = np.zeros((model.n, model.n), dtype=np.complex128)
        for beta in (range(M) if betas is None else betas(mu)):
            acc += eom_term(model, gammas, G, h, E, lam, mu, beta)
        out.append(2.0 * np.real(np.conj(lt[mu]) * c[mu] * acc))
    return out


# ---------------------------------------------------------------------------
# Integrator (App. A)
# ---------------------------------------------------------------------------


def orthogonal_step(Gm, dG, ds):
    """Gamma <- R Gamma R^T with R = exp{(ds/4)[Gamma, dGamma]} (Eq. ExpStep)."""
    X = 0.25 * ds * (Gm @ dG - dG @ Gm)
    R = scipy.linalg.expm(X)
    out = R @ Gm @ R.T
    return 0.5 * (out - out.T)


def purify(Gm):
    """Canonical-form renormalisation of App. A (Eq. CM-normal-form with every
    lambda_j set to 1): the orthogonal polar factor Gamma (Gamma^T Gamma)^{-1/2}."""
    w, V = np.linalg.eigh(Gm.T @ Gm)
    P = Gm @ (V / np.sqrt(w)) @ V.T
    return 0.5 * (P - P.T)


def euler_step(Gm, dG, ds):
    """First-order step of Eq. (RKstep) followed by the canonical-form
    renormalisation of App. A."""
    return purify(Gm + ds * dG)


# ---------------------------------------------------------------------------
# One step and the energy (Sec. III C)
# ---------------------------------------------------------------------------


def energy(model, gammas):
    """Energy of the current states with optimal amplitudes (Eq. eigLambda).
    Returns (E, lambda, G, h)."""
    G, h = gram_and_hamiltonian(model, gammas)
    E, lam = solve_amplitudes(G, h)
    return E, lam, G, h


def sgs_step(model, gammas, ds, mode=C_INVERSE, purify_each=True):
    """One step of Sec. III C: pairs -> amplitudes -> EOM -> orthogonal update
    -> re-purification.  Returns (E before the update, lambda, new gammas)."""
    E, lam, G, h = energy(model, gammas)
    dGs = eom(model, gammas, G, h, E, lam, mode)
    new = []
    for Gm, dG in zip(gammas, dGs):
        g = orthogonal_step(Gm, dG, ds)
        new.append(purify(g) if purify_each else g)
    return E, lam, new


def run(model, gammas, ds, n_steps, mode=C_INVERSE):
    """n_steps of sgs_step; returns (energies, lambda, gammas)."""
    Es = []
    lam = None
    for _ in range(n_steps):
        E, lam, gammas = sgs_step(model, gammas, ds, mode)
        Es.append(E)
    return np.array(Es), lam, gammas


def euler_run(model, gammas, ds, n_steps, mode=C_INVERSE):
    """n_steps with the first-order integrator of Eq. (RKstep) in place of the
    orthogonal step; returns (energies, lambda, gammas)."""
    Es = []
    lam = None
    for _ in range(n_steps):
        E, lam, G, h = energy(model, gammas)
        dGs = eom(model, gammas, G, h, E, lam, mode)
        gammas = [euler_step(Gm, dG, ds) for Gm, dG in zip(gammas, dGs)]
        Es.append(E)
    return np.array(Es), lam, gammas


# ---------------------------------------------------------------------------
# Rank growth (Sec. III C)
# ---------------------------------------------------------------------------


def add_state(gammas, K, src):
    """Append the state Q Gamma_src Q^T, Q = exp(K) with K antisymmetric (a
    special orthogonal Q; the paper draws it at random close to the identity
    and applies it to a state of high amplitude)."""
    Q = scipy.linalg.expm(K)
    g = Q @ gammas[src] @ Q.T
    return list(gammas) + [0.5 * (g - g.T)]


def grow(model, gammas, ds, steps_per_rank, Ks, mode=C_INVERSE):
    """The paper's schedule: evolve steps_per_rank steps, then add one state
    copied (through exp(K_j)) from the state of largest |lambda_mu| at the last
    amplitude solve, once per K_j; finish with steps_per_rank steps at the final
    rank.  Returns (energies of every step, final gammas)."""
    Es = []
    for K in list(Ks) + [None]:
        E, lam, gammas = run(model, gammas, ds, steps_per_rank, mode)
        Es.extend(E)
        if K is None:
            break
        gammas = add_state(gammas, K, int(np.argmax(np.abs(lam))))
    return np.array(Es), gammas


# ---------------------------------------------------------------------------
# Hamiltonian variance (Eq. residual) and the energy extrapolation (Sec. IV A)
# ---------------------------------------------------------------------------
#
# H = e + H2 + H4 with H2 = i sum_kl A_kl c_k c_l and H4 = sum_m v_m c_m0 c_m1 c_m2 c_m3
# (monomials with increasing indices).  In the transition "state" of a pair the
# ordered contraction of c_x (left) with c_y (right) is g_xy = delta_xy + i Delta_xy,
# and by Wick's theorem a product of Majoranas (repeats allowed) is the Pfaffian
# of the ordered contractions.  Summing the Wick terms of H^2 over the quadratic
# indices in matrix form:
#   <H2>      = T = Tr(A Delta)
#   <H2 H2>   = T^2 - 2 tr(A^2) - 2 tr(A Delta A Delta)
#   <H2 H4_m> = T Pf4_m - i dPf4_m[C],   C  = B - B^T,   B  = g^T A g
#   <H4_m H2> = T Pf4_m - i dPf4_m[C'],  C' = B' - B'^T, B' = g A g^T
#   <H4_m H4_m'> = Pf8 of the ordered contractions of (m, m')
# with Pf4_m the Pfaffian of g on the monomial's indices and dPf4_m[C] its
# derivative in the direction C (C on one pair of indices, g on the other).


def canonical_quartic(model):
    """The quartic part as monomials with increasing indices: coefficient of
    c_k c_l c_p c_q (k < l < p < q) = 24 U_klpq of the antisymmetric U."""
    return [(idx, 24.0 * v) for idx, v in model.quartic if list(idx) == sorted(idx)]


def _ordered_contractions(g, idx):
    m = len(idx)
    X = np.zeros((m, m), dtype=np.complex128)
    for a in range(m):
        for b in range(a + 1, m):
            X[a, b] = g[idx[a], idx[b]]
            X[b, a] = -X[a, b]
    return X


def _pf4(X):
    return X[0, 1] * X[2, 3] - X[0, 2] * X[1, 3] + X[0, 3] * X[1, 2]


def _dpf4(X, C):
    return (C[0, 1] * X[2, 3] + X[0, 1] * C[2, 3] - C[0, 2] * X[1, 3] - X[0, 2] * C[1, 3]
            + C[0, 3] * X[1, 2] + X[0, 3] * C[1, 2])


def hamiltonian_square_density(model, Dlt):
    """<H^2> in the transition state with matrix Dlt: <phi_a|H^2|phi_b> / G_ab
    for Dlt = Delta^{b,a} (Gamma_a itself for a = b).  Quadratic and quartic
    terms only."""
    if model.higher:
        raise NotImplementedError("the variance covers quadratic and quartic terms")
    A = model.A
    n = model.n
    e = model.e_const
    g = np.eye(n) + 1j * Dlt
    T = np.trace(A @ Dlt)
    X = A @ Dlt
    h22 = T * T - 2.0 * np.trace(A @ A) - 2.0 * np.trace(X @ X)
    B = g.T @ A @ g
    Bp = g @ A @ g.T
    C, Cp = B - B.T, Bp - Bp.T
    mons = canonical_quartic(model)
    Q = h24 = h42 = h44 = 0.0 + 0.0j
    for idx, v in mons:
        Xm = _ordered_contractions(g, idx)
        p4 = _pf4(Xm)
        Q += v * p4
        h24 += v * (T * p4 - 1j * _dpf4(Xm, C[np.ix_(idx, idx)]))
        h42 += v * (T * p4 - 1j * _dpf4(Xm, Cp[np.ix_(idx, idx)]))
        for idx2, v2 in mons:
            h44 += v * v2 * pfaffian(_ordered_contractions(g, list(idx) + list(idx2)))
    return e * e + 2.0 * e * (T + Q) + h22 + h24 + h42 + h44


def variance(model, gammas):
    """delta_H^2 = <psi|H^2|psi> - <psi|H|psi>^2 (Eq. residual) for the optimal
    amplitudes normalised to <psi|psi> = 1.  Returns (E, delta_H^2)."""
    E, lam, G, h = energy(model, gammas)
    M = len(gammas)
    tot = 0.0 + 0.0j
    for a in range(M):
        for b in range(M):
            D = gammas[a].astype(np.complex128) if a == b else transition_matrix(gammas[b], gammas[a])
            tot += np.conj(lam[a]) * lam[b] * G[a, b] * hamiltonian_square_density(model, D)
    return E, float(tot.real) - E * E


def extrapolate_energy(energies, variances, var_max=2e-5):
    """Linear fit E = E* + k delta_H^2 over the points with delta_H^2 < var_max
    (Sec. IV A); returns (E*, standard error of the intercept)."""
    E = np.asarray(energies, dtype=float)
    v = np.asarray(variances, dtype=float)
    keep = v < var_max
    E, v = E[keep], v[keep]
    if len(E) < 3:
        raise ValueError("need at least three points below var_max")
    Xd = np.stack([np.ones_like(v), v], 1)
    coef, res, _, _ = np.linalg.lstsq(Xd, E, rcond=None)
    r = E - Xd @ coef
    s2 = float(r @ r) / (len(E) - 2)
    cov = s2 * np.linalg.inv(Xd.T @ Xd)
    return float(coef[0]), float(math.sqrt(cov[0, 0]))


# ---------------------------------------------------------------------------
# Observables: spin-spin correlators (Eq. Cr, Eq. K2CK)
# ---------------------------------------------------------------------------
#
# Operators are Majorana polynomials {(i1 < i2 < ...): coefficient}.  The
# expectation of a monomial c_I (distinct, increasing indices) in the
# transition "state" with matrix Delta is the Pfaffian of the sub-block of
# i Delta on I (Sec. III B: n-point elements are Pfaffians of n x n
# sub-matrices), 1 for the empty monomial.


def _mono_mul(a, b):
    """Product of two normal-ordered Majorana monomials: (sign, monomial)."""
    seq = list(a) + list(b)
    sign = 1
    # bubble sort with anticommutation signs, then cancel c_p c_p = 1
    for i in range(len(seq)):
        for j in range(len(seq) - 1 - i):
            if seq[j] > seq[j + 1]:
                seq[j], seq[j + 1] = seq[j + 1], seq[j]
                sign = -sign
    out = []
    for x in seq:
        if out and out[-1] == x:
            out.pop()
        else:
            out.append(x)
    return sign, tuple(out)


def poly_mul(P, Q):
    R = {}
    for a, ca in P.items():
        for b, cb in Q.items():
            s, m = _mono_mul(a, b)
            R[m] = R.get(m, 0.0) + s * ca * cb
    return {m: c for m, c in R.items() if c != 0}


def poly_add(P, Q, q=1.0):
    R = dict(P)
    for m, c in Q.items():
        R[m] = R.get(m, 0.0) + q * c
    return {m: c for m, c in R.items() if c != 0}


def _annihilator(mode):
    """a_m = (c_{2m} + i c_{2m+1}) / 2 as a polynomial."""
    return {(2 * mode,): 0.5, (2 * mode + 1,): 0.5j}


def _creator(mode):
    return {(2 * mode,): 0.5, (2 * mode + 1,): -0.5j}


def spin_operators(site):
    """S^x, S^y, S^z of a spinful site (modes 2 site + sigma) from
    S = 1/2 sum_ss' d^dag_s sigma_ss' d_s' (Eq. Cr), as Majorana polynomials."""
    up, dn = 2 * site, 2 * site + 1
    updn = poly_mul(_creator(up), _annihilator(dn))
    dnup = poly_mul(_creator(dn), _annihilator(up))
    nu = poly_mul(_creator(up), _annihilator(up))
    nd = poly_mul(_creator(dn), _annihilator(dn))
    Sx = {m: 0.5 * c for m, c in poly_add(updn, dnup).items()}
    Sy = {m: -0.5j * c for m, c in poly_add(updn, dnup, -1.0).items()}
    Sz = {m: 0.5 * c for m, c in poly_add(nu, nd, -1.0).items()}
    return Sx, Sy, Sz


def spin_dot(site_a, site_b):
    A, B = spin_operators(site_a), spin_operators(site_b)
    out = {}
    for x, y in zip(A, B):
        out = poly_add(out, poly_mul(x, y))
    return out


def poly_expectation(P, Dlt):
    """<O>_t = sum_I coeff_I Pf((i Delta)[I, I])."""
    tot = 0.0 + 0.0j
    for m, c in P.items():
        if len(m) == 0:
            tot += c
        elif len(m) % 2 == 0:
            idx = list(m)
            tot += c * pfaffian(1j * Dlt[np.ix_(idx, idx)])
    return tot


def sgs_expectation(P, gammas, lam, G):
    """<psi|O|psi> = sum_ab conj(lambda_a) lambda_b <phi_a|O|phi_b>, with
    <phi_a|O|phi_b> = G_ab <O>_t evaluated on Delta^{b,a} (Sec. III B)."""
    M = len(gammas)
    tot = 0.0 + 0.0j
    for a in range(M):
        for b in range(M):
            D = gammas[a].astype(np.complex128) if a == b else transition_matrix(gammas[b], gammas[a])
            tot += np.conj(lam[a]) * lam[b] * G[a, b] * poly_expectation(P, D)
    return tot


def spin_correlator(gammas, lam, G, sites):
    """C(r) = <S(0) . S(r)> for the impurity site 0 and each site in ``sites``."""
    return np.array([np.real(sgs_expectation(spin_dot(0, s), gammas, lam, G)) for s in sites])


def two_channel_correlator(gammas, lam, G, distances, n_channels=2):
    """K(r) = sum_alpha <S_imp . S_alpha(r)> (Eq. K2CK) with the interleaved
    site order of anderson_chain: channel alpha, chain site r -> 1 + (r-1) n_ch + alpha."""
    out = []
    for r in distances:
        tot = 0.0
        for al in range(n_channels):
            tot += np.real(sgs_expectation(spin_dot(0, 1 + (r - 1) * n_channels + al), gammas, lam, G))
        out.append(tot)
    return np.array(out)


# ---------------------------------------------------------------------------
# Renyi-2 entropy of the leading modes (App. B, Eqs. S2_SGS, T_tensor,
# TrArho2_final)
# ---------------------------------------------------------------------------


def _m_block(Ga, Gb, sl):
    """M_J^{a,b} = [[Gamma_J^a, i 1], [-i 1, Gamma_J^b]] (Eq. MB)."""
    m = sl.stop - sl.start
    I = np.eye(m)
    return np.block([[Ga[sl, sl], 1j * I], [-1j * I, Gb[sl, sl]]])


def renyi2_trace_term(Ga, Gb, Gc, Gd, n_modes_A):
    """I^{a,b}_{c,d} = Tr_A(Tr_B(rho_a rho_b) Tr_B(rho_c rho_d)) by Eq. TrArho2_final:
    2^{N_B}/8^N Pf[M_B^{ab}] Pf[M_B^{cd}] Pf[M_A^{cd} + Sigma_A^{cd}]
    Pf[M_A^{ab} + Sigma_A^{ab} + sigma_A^{dc}], with Sigma_A (Eq. MB) and
    sigma_A^{dc} = -X (M_A^{cd} + Sigma_A^{cd})^{-1} X, X = [[-1, 1], [1, -1]]."""
    n = Ga.shape[0]
    N = n // 2
    NA = n_modes_A
    NB = N - NA
    A = slice(0, 2 * NA)
    B = slice(2 * NA, n)

    def sigma_A(G1, G2):
        if NB == 0:
            return np.zeros((4 * NA, 4 * NA), dtype=np.complex128)
        Z = np.zeros((2 * NA, 2 * NB))
        GAB = np.block([[G1[A, B], Z], [Z, G2[A, B]]])
        MB = _m_block(G1, G2, B)
        return GAB @ np.linalg.solve(MB, GAB.T)

    pfB_ab = pfaffian(_m_block(Ga, Gb, B)) if NB > 0 else 1.0
    pfB_cd = pfaffian(_m_block(Gc, Gd, B)) if NB > 0 else 1.0
    MA_ab = _m_block(Ga, Gb, A) + sigma_A(Ga, Gb)
    MA_cd = _m_block(Gc, Gd, A) + sigma_A(Gc, Gd)
    I2 = np.eye(2 * NA)
    X = np.block([[-I2, I2], [I2, -I2]])
    sig = -X @ np.linalg.solve(MA_cd, X)
    return 2.0 ** NB / 8.0 ** N * pfB_ab * pfB_cd * pfaffian(MA_cd) * pfaffian(MA_ab + sig)


def renyi2(gammas, lam, G, n_modes_A):
    """S_2(A) = -ln sum_abcd T^{ab}_{cd} (Eq. S2_SGS) with
    T^{ab}_{cd} = lambda_a conj(lambda_b) lambda_c conj(lambda_d) I^{ab}_{cd} / (G_ab G_cd)
    (Eq. T_tensor); A = the first n_modes_A fermion modes."""
    M = len(gammas)
    tot = 0.0 + 0.0j
    for a in range(M):
        for b in range(M):
            for c in range(M):
                for d in range(M):
                    I = renyi2_trace_term(gammas[a], gammas[b], gammas[c], gammas[d], n_modes_A)
                    tot += lam[a] * np.conj(lam[b]) * lam[c] * np.conj(lam[d]) * I / (G[a, b] * G[c, d])
    return float(-math.log(tot.real))
