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


def overlap_error_bars(ga, gb, g0, delta, rtol=1e-10):
    """Bars for one pair element G_ab = |G_ab| e^{i phi} computed twice (two
    implementations, two roundings), from the conditioning of the two
    factorisations it comes from (Sec. II B: the magnitude from
    log|det(Gamma_a + Gamma_b)|, the phase from Pf(Gamma_0 + Delta^{a,b})).

    A backward-stable factorisation of X returns the log-determinant of
    X + dX with |dX|_2 <= n u |X|_2, and to first order
    d log det X = tr(X^-1 dX), so |d log|det X|| <= n u |X|_2 sum_i 1/sigma_i(X).
    The log of a Pfaffian moves by half that.  With two computations:

        | log|G_gpu| - log|G_ref| | <= rtol + n u |S|_2 sum 1/sigma_i(S)
        | arg(G_gpu / G_ref) |      <= rtol + n u |Y|_2 sum 1/sigma_i(Y)

    S = Gamma_a + Gamma_b, Y = Gamma_0 + Delta^{a,b} (no phase Pfaffian for
    a pair with the reference state 0: pass g0 = None).  The bound is worst
    case over the direction of the rounding, so it is loose for a nearly
    singular Y; nothing in it is fitted to a measured result.
    Returns (magnitude bar, phase bar)."""
    S = ga + gb
    n = S.shape[0]
    sv = np.linalg.svd(S, compute_uv=False)
    mag = rtol + n * U * sv[0] * np.sum(1.0 / sv)
    ph = rtol
    if g0 is not None:
        sy = np.linalg.svd(g0 + delta, compute_uv=False)
        ph += n * U * sy[0] * np.sum(1.0 / sy)
    return mag, ph
