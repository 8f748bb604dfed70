"""Fock-space brute force for tiny systems (N <= 10 fermion modes).

Independent of the oracle: builds Jordan-Wigner fermion operators, explicit
Gaussian state vectors, the many-body Hamiltonian from creation/annihilation
operators, and evaluates overlaps, matrix elements, equations of motion,
correlators and Renyi entropies directly on vectors.  Used only to pin the
oracle.
"""
from __future__ import annotations

import functools

import numpy as np
import scipy.sparse as sp


@functools.lru_cache(maxsize=None)
def annihilators(N: int):
    """a_j, j = 0..N-1, as sparse 2^N x 2^N matrices (Jordan-Wigner, mode 0 is
    the most significant tensor factor; basis state |n_0 n_1 ...>)."""
    I = sp.identity(2, format="csr", dtype=np.complex128)
    Z = sp.csr_matrix(np.diag([1.0, -1.0]).astype(np.complex128))
    lower = sp.csr_matrix(np.array([[0.0, 1.0], [0.0, 0.0]], dtype=np.complex128))  # |0><1|
    ops = []
    for j in range(N):
        mats = [Z] * j + [lower] + [I] * (N - j - 1)
        a = mats[0]
        for m in mats[1:]:
            a = sp.kron(a, m, format="csr")
        ops.append(a.tocsr())
    return tuple(ops)


@functools.lru_cache(maxsize=None)
def majoranas(N: int):
    """c_{2j} = a_j + a_j^dag, c_{2j+1} = -i (a_j - a_j^dag)."""
    out = []
    for a in annihilators(N):
        ad = a.conj().T.tocsr()
        out.append((a + ad).tocsr())
        out.append((-1j * (a - ad)).tocsr())
    return tuple(out)


def number_op(N, j):
    a = annihilators(N)[j]
    return (a.conj().T @ a).tocsr()


def gaussian_vector(Gamma, ref=None):
    """Ground state of the parent Hamiltonian (i/2) sum_kl Gamma_kl c_k c_l,
    whose unique ground state has covariance Gamma when Gamma^2 = -1.
    If ``ref`` is given, the phase is fixed so that <ref|phi> > 0."""
    n = Gamma.shape[0]
    N = n // 2
    c = majoranas(N)
    H = sp.csr_matrix((2 ** N, 2 ** N), dtype=np.complex128)
    for k in range(n):
        for l in range(n):
            if Gamma[k, l] != 0.0:
                H = H + (0.5j * Gamma[k, l]) * (c[k] @ c[l])
    w, v = np.linalg.eigh(H.toarray())
    phi = v[:, 0]
    if ref is not None:
        ov = np.vdot(ref, phi)
        phi = phi * (abs(ov) / ov)
    return phi


def covariance_of(phi):
    N = int(round(np.log2(phi.shape[0])))
    c = majoranas(N)
    n = 2 * N
    G = np.zeros((n, n))
    for k in range(n):
        ck = c[k] @ phi
        for l in range(n):
            if k != l:
                G[k, l] = np.real(-1j * np.vdot(phi, c[k] @ (c[l] @ phi)))
    return G


def hamiltonian_anderson(n_sites_per_channel_bath, U, eps_d, V, t=1.0, mu=0.0, n_channels=1):
    """Anderson impurity built from fermion operators: impurity site 0, bath
    chains of ``n_sites_per_channel_bath`` sites per channel, channels
    interleaved (site 1 + (r-1)*n_channels + c), mode 2*site + spin.
    H = sum_sigma [eps_d n_0sigma - V sum_c (d0^dag d_{c,1} + h.c.)
        - t sum_c sum_r (d_{c,r-1}^dag d_{c,r} + h.c.) - mu sum n_bath]
        + U n_0up n_0dn."""
    L = n_sites_per_channel_bath
    n_sites = 1 + n_channels * L
    N = 2 * n_sites
    a = annihilators(N)
    ad = [x.conj().T.tocsr() for x in a]

    def site(c, r):
        return 1 + (r - 1) * n_channels + c

    H = sp.csr_matrix((2 ** N, 2 ** N), dtype=np.complex128)
    for s in range(2):
        H = H + eps_d * (ad[s] @ a[s])
        for c in range(n_channels):
            m = 2 * site(c, 1) + s
            H = H - V * (ad[s] @ a[m] + ad[m] @ a[s])
            for r in range(1, L + 1):
                m = 2 * site(c, r) + s
                H = H - mu * (ad[m] @ a[m])
                if r >= 2:
                    p = 2 * site(c, r - 1) + s
                    H = H - t * (ad[p] @ a[m] + ad[m] @ a[p])
    H = H + U * (ad[0] @ a[0]) @ (ad[1] @ a[1])
    return H.tocsr()


def ground_energy(H):
    d = H.shape[0]
    if d <= 4096:
        return float(np.linalg.eigvalsh(H.toarray())[0])
    import scipy.sparse.linalg as sla
    return float(sla.eigsh(H, k=1, which="SA")[0][0])


def gram(vecs):
    return np.array([[np.vdot(a, b) for b in vecs] for a in vecs])


def hmat(vecs, H):
    Hv = [H @ v for v in vecs]
    return np.array([[np.vdot(a, hb) for hb in Hv] for a in vecs])


def lowest_amplitudes(G, h):
    """Lowest generalised eigenpair of h x = E G x by Cholesky reduction
    (a different route from the oracle's canonical orthogonalisation)."""
    L = np.linalg.cholesky(G)
    Li = np.linalg.inv(L)
    Hs = Li @ h @ Li.conj().T
    e, V = np.linalg.eigh(0.5 * (Hs + Hs.conj().T))
    x = Li.conj().T @ V[:, 0]
    return float(e[0]), x


def eom_bruteforce(vecs, lam, H, mode="inverse"):
    """d Gamma^mu / ds from the state-level flow of Sec. III A:
    d phi_mu = -B_mu phi_mu, B_mu = c_mu Pi_perp H |psi><psi| + h.c., and
    d Gamma_kl = -<phi| i c_k c_l |d phi> + c.c."""
    M = len(vecs)
    N = int(round(np.log2(vecs[0].shape[0])))
    c = majoranas(N)
    n = 2 * N
    G = gram(vecs)
    Gi = np.linalg.inv(G)
    psi = sum(lam[m] * vecs[m] for m in range(M))
    Hpsi = H @ psi
    # Pi_perp H psi
    coef = Gi @ np.array([np.vdot(v, Hpsi) for v in vecs])
    proj = Hpsi - sum(coef[a] * vecs[a] for a in range(M))
    out = []
    for mu in range(M):
        lt = np.vdot(vecs[mu], psi)
        z = lam[mu] * np.conj(lt)
        cm = 1.0 / z if mode == "inverse" else np.conj(z) / abs(z)
        # B_mu |phi_mu> = c_mu Pi H |psi> <psi|phi_mu> + c_mu^* |psi><psi| H Pi |phi_mu>,
        # and Pi |phi_mu> = 0
        dphi = -cm * np.conj(lt) * proj
        dG = np.zeros((n, n))
        for k in range(n):
            for l in range(n):
                if k != l:
                    x = np.vdot(vecs[mu], c[k] @ (c[l] @ dphi))
                    dG[k, l] = 2.0 * np.real(-1j * x)
        out.append(dG)
    return out


def spin_ops(N, site):
    """(Sx, Sy, Sz) of a spinful site (modes 2*site, 2*site+1)."""
    a = annihilators(N)
    up, dn = a[2 * site], a[2 * site + 1]
    upd, dnd = up.conj().T, dn.conj().T
    Sp = upd @ dn
    Sm = dnd @ up
    Sz = 0.5 * (upd @ up - dnd @ dn)
    Sx = 0.5 * (Sp + Sm)
    Sy = -0.5j * (Sp - Sm)
    return Sx.tocsr(), Sy.tocsr(), Sz.tocsr()


def spin_spin(psi, N, s0, s1):
    A = spin_ops(N, s0)
    B = spin_ops(N, s1)
    psi = psi / np.linalg.norm(psi)
    return float(np.real(sum(np.vdot(psi, a @ (b @ psi)) for a, b in zip(A, B))))


def renyi2_leading_modes(psi, n_modes_A):
    """S_2 of the first ``n_modes_A`` modes (leading Jordan-Wigner factors).
    For a parity-definite state the Jordan-Wigner strings of the leading
    modes act inside A, so this is the fermionic reduced density matrix."""
    N = int(round(np.log2(psi.shape[0])))
    psi = psi / np.linalg.norm(psi)
    m = psi.reshape(2 ** n_modes_A, 2 ** (N - n_modes_A))
    rho = m @ m.conj().T
    return float(-np.log(np.real(np.trace(rho @ rho))))
