"""Conditioning of the amplitude problem h lambda = E G lambda (Eq. eigLambda)
and the tolerance it implies for dGamma^mu (test infrastructure).

The decoupling constant of Sec. III A makes dGamma^mu proportional to
1 / lambda_mu (c_mu = [lambda_mu conj(lt_mu)]^-1), or to the phase of lambda_mu
(the phase form of c_mu).  Either way a perturbation delta lambda_mu of the
solved amplitude changes dGamma^mu by |delta lambda_mu| / |lambda_mu| relative
to first order.  Two implementations solve the problem from their own (G, h)
with their own roundings, so their amplitudes differ by (first-order
perturbation of a generalized Hermitian eigenvector, normalised to
lambda^dag G lambda = 1)

    delta lambda = -S (delta h - E delta G) lambda - (1/2)(lambda^dag delta G lambda) lambda,
    S = sum_{k > 0} lambda_k lambda_k^dag / (E_k - E_0),

where delta G, delta h are the differences of the two inputs plus the
backward errors of the two solves.  A backward-stable solve of the real 2M x
2M embedding perturbs (G, h) by at most about 2M u of their norms; the bound
takes that for each of the two solves.  dGamma^mu is then held to
1e-10 + 2 |delta lambda_mu| / |lambda_mu| relative (the factor 2 covers the
second-order terms and the other amplitudes' share of the sum over beta).
Nothing here is fitted to a measured result: the inputs are the oracle's
(G, h, E, lambda) and the two implementations' (G, h)."""
import numpy as np

U = 2.0 ** -53


def amplitude_sensitivity(G, h):
    """S of the first-order formula, in the retained space of the canonical
    orthogonalisation (eigenvalues of G below 1e-12 of the largest dropped, as
    the oracle does)."""
    w, V = np.linalg.eigh(G)
    keep = w > 1e-12 * w.max()
    X = V[:, keep] / np.sqrt(w[keep])
    ev, Y = np.linalg.eigh(X.conj().T @ h @ X)
    Z = X @ Y
    inv = np.zeros_like(ev)
    inv[1:] = 1.0 / (ev[1:] - ev[0])
    return (Z * inv) @ Z.conj().T


def lambda_error_bound(Go, ho, Eo, lo, Gg, hg):
    """Per-state bound on |lambda_mu| differences between two solves: one from
    (Go, ho) with solution (Eo, lo), one from (Gg, hg)."""
    M = len(lo)
    S = amplitude_sensitivity(Go, ho)
    r = np.linalg.norm(((hg - ho) - Eo * (Gg - Go)) @ lo)
    eta = 2 * (2 * M) * U * (np.linalg.norm(ho, 2) + abs(Eo) * np.linalg.norm(Go, 2)) * np.linalg.norm(lo)
    norm_term = 0.5 * (np.linalg.norm(Gg - Go, 2) + 2 * (2 * M) * U * np.linalg.norm(Go, 2)) * np.linalg.norm(lo) ** 2
    return np.linalg.norm(S, axis=1) * (r + eta) + norm_term * np.abs(lo)


def dgamma_rtol(bound, lo, mu, base=1e-10):
    """Relative tolerance of dGamma^mu (to its largest entry)."""
    return base + 2.0 * bound[mu] / max(abs(lo[mu]), 1e-300)
