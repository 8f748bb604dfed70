"""The algebra of the per-state update (App. A, Eq. ExpStep) as the CUDA path
runs it (CPU): numpy transcriptions of

- the FP64 form: X = (ds/4)(Y - Y^T) from Y = Gamma dGamma, the squaring count
  (||X 2^-s||_F <= 1/8), the degree-10 Taylor polynomial by Paterson-Stockmeyer
  in blocks of three, the squarings, R Gamma R^T and one Newton-Schulz
  iteration X <- 1.5 X + 0.5 X (X X);
- the mixed forms' increment form: E = R - I by Horner on transposes
  (Q_d = I - X_s / d, Q_j = I + (1/j) Q_{j+1} X_s^T, E^T = Q_2 X_s^T), the
  squarings E^T <- 2 E^T + E^T E^T, and Gamma' = Gamma + F - F^T + (G - G^T)/2
  with F = E Gamma, G = F E^T;

against the oracle's orthogonal step (scipy's expm) and the exact polar factor.
Variants with a dropped Taylor block, a Horner recurrence on X_s in place of
its transpose, or squarings without the 2E term are caught."""
import math
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import Polynomial

import sgs_inputs as inp
from oracle import sgs_oracle as orc

THETA = 0.125
MAX_SQUARINGS = 14


def squarings(X):
    nrm = np.sqrt((X * X).sum())
    s = 0
    while nrm * 2.0 ** -s > THETA and s < 64:
        s += 1
    return min(s, MAX_SQUARINGS)


def taylor_coefficients():
    cf = [1.0]
    for k in range(1, 12):
        cf.append(cf[-1] / k)
    cf[11] = 0.0                      # degree 10: the top coefficient of the last block is unused
    return cf


def skew_product(A, B):
    """A product whose result is antisymmetric, computed as the SKEW mode does: the strictly lower
    triangle, mirrored with a sign, zero diagonal."""
    L = np.tril(A @ B, -1)
    return L - L.T


def paterson_stockmeyer(Xs, one, mul, skew_mul, drop_block=None):
    """p(Xs) = sum_{k <= 10} Xs^k / k! in blocks of three: B = c10 Xs + c9, then
    B <- B Y + c_{3j+2} Xs^2 + c_{3j+1} Xs + c_{3j} for j = 2, 1, 0 with Y = Xs^3."""
    cf = taylor_coefficients()
    X2 = mul(Xs, Xs)
    X3 = skew_mul(X2, Xs)
    B = cf[10] * Xs + cf[9] * one
    for j in (2, 1, 0):
        if j == drop_block:
            continue
        B = mul(B, X3) + cf[3 * j + 2] * X2 + cf[3 * j + 1] * Xs + cf[3 * j] * one
    return B


def _ns(X, XX):
    # C = 0.5 X (X X) + 1.5 X, as the SKEW epilogue writes it (lower triangle, mirrored)
    L = np.tril(0.5 * (X @ XX) + 1.5 * X, -1)
    return L - L.T


def fp64_update(Gm, dG, ds, drop_block=None):
    n = Gm.shape[0]
    Y = Gm @ dG
    X = 0.25 * ds * (Y - Y.T)
    s = squarings(X)
    Xs = 2.0 ** -s * X
    R = paterson_stockmeyer(Xs, np.eye(n), lambda a, b: a @ b, skew_product, drop_block)
    for _ in range(s):
        R = R @ R
    T = R @ Gm
    L = np.tril(T @ R.T, -1)
    return _ns(L - L.T, (L - L.T) @ (L - L.T)), s


def increment_update(Gm, dG, ds, degree=6, transposed=True, two_e=True):
    n = Gm.shape[0]
    Y = Gm @ dG
    X = 0.25 * ds * (Y - Y.T)
    s = squarings(X)
    Xs = 2.0 ** -s * X
    XT = Xs.T if transposed else Xs
    Q = np.eye(n) + XT / degree                            # Q_d = P_d^T = I + X_s^T / d = I - X_s / d
    for j in range(degree - 1, 1, -1):
        Q = np.eye(n) + (1.0 / j) * (Q @ XT)
    ET = Q @ XT
    for _ in range(s):
        ET = ET @ ET + (2.0 * ET if two_e else 0.0)
    E = ET.T
    F = E @ Gm
    G = F @ ET
    return Gm + (F - F.T) + 0.5 * (G - G.T), E, X


def _state_and_direction(seed, n_bath=3):
    model = orc.anderson_model(n_bath, 2.0, -1.0, 0.5)
    rng = np.random.default_rng(seed)
    gammas = [inp.random_pure_gamma(model.N, rng) for _ in range(3)]
    E, lam, G, h = orc.energy(model, gammas)
    dG = orc.eom(model, gammas, G, h, E, lam)
    return gammas[1], dG[1]


def test_paterson_stockmeyer_is_the_degree_10_taylor_polynomial():
    """Run on polynomials in one variable, the evaluation yields exactly the coefficients 1/k!,
    k <= 10; a dropped block is caught."""
    x = Polynomial([0.0, 1.0])
    p = paterson_stockmeyer(x, Polynomial([1.0]), lambda a, b: a * b, lambda a, b: a * b)
    ref = [1.0 / math.factorial(k) for k in range(11)]
    assert np.allclose(p.coef, ref, rtol=1e-15, atol=0.0) and len(p.coef) == 11
    bad = paterson_stockmeyer(x, Polynomial([1.0]), lambda a, b: a * b, lambda a, b: a * b, drop_block=1)
    assert not (len(bad.coef) == 11 and np.allclose(bad.coef, ref, rtol=1e-12, atol=0.0))


def test_taylor_truncation_below_3e_18():
    """With ||X_s|| <= 1/8 the terms beyond degree 10 sum to below 3e-18 (Lagrange remainder
    bounded by the series tail, in exact rationals)."""
    theta = Fraction(1, 8)
    tail = sum(theta ** k / math.factorial(k) for k in range(11, 40))
    assert tail < Fraction(3, 10 ** 18)
    # and degree 6 (the mixed forms) truncates below 1e-10 relative to ||E|| >= ||X_s|| (1 - ||X_s||)
    tail6 = sum(theta ** k / math.factorial(k) for k in range(7, 40))
    assert tail6 / (theta * (1 - theta)) < Fraction(1, 10 ** 9)


@pytest.mark.parametrize("norm,s", [(0.1, 0), (0.125, 0), (0.13, 1), (1.0, 3), (1.0001, 4), (1e9, 14)])
def test_squaring_count(norm, s):
    A = np.zeros((4, 4))
    A[0, 1], A[1, 0] = 1.0, -1.0
    X = A * norm / np.sqrt(2.0)
    assert squarings(X) == s


@pytest.mark.parametrize("ds,n_sq", [(0.01, 0), (0.05, 1), (2.0, 6), (40.0, 11)])
def test_fp64_update_equals_the_oracle_step(ds, n_sq):
    """The transcription equals the oracle's orthogonal step followed by the polar factor, with and
    without squarings; one Newton-Schulz iteration suffices because R is orthogonal to rounding."""
    Gm, dG = _state_and_direction(11)
    out, s = fp64_update(Gm, dG, ds)
    ref = orc.purify(orc.orthogonal_step(Gm, dG, ds))
    assert s == n_sq
    assert np.abs(out - ref).max() < 1e-13
    assert np.abs(out + out.T).max() == 0.0
    assert np.abs(out @ out + np.eye(len(out))).max() < 1e-13


def test_fp64_update_with_a_dropped_block_is_caught():
    Gm, dG = _state_and_direction(12)
    out, _ = fp64_update(Gm, dG, 2.0, drop_block=0)
    ref = orc.purify(orc.orthogonal_step(Gm, dG, 2.0))
    assert np.abs(out - ref).max() > 1e-6


@pytest.mark.parametrize("ds", [0.05, 2.0])
def test_increment_form_equals_the_exponential(ds):
    """E = R - I to 1e-9 of ||E|| (degree 6), and Gamma + F - F^T + (G - G^T)/2 = R Gamma R^T for
    that R to rounding; after the polar factor the step equals the oracle's to the truncation."""
    Gm, dG = _state_and_direction(13)
    G1, E, X = increment_update(Gm, dG, ds)
    from scipy.linalg import expm
    Eref = expm(X) - np.eye(len(X))
    assert np.abs(E - Eref).max() < 1e-9 * np.abs(Eref).max()
    R = np.eye(len(X)) + E
    direct = R @ Gm @ R.T
    assert np.abs(G1 - 0.5 * (direct - direct.T)).max() < 1e-14
    ref = orc.purify(orc.orthogonal_step(Gm, dG, ds))
    assert np.abs(orc.purify(G1) - ref).max() < 1e-8


def test_increment_form_variants_are_caught():
    """A recurrence on X_s where its transpose belongs (the operand's K-major form misread) and
    squarings without the 2E term both leave the exponential."""
    Gm, dG = _state_and_direction(14)
    from scipy.linalg import expm
    for kw in ({"transposed": False}, {"two_e": False}):
        _, E, X = increment_update(Gm, dG, 2.0, **kw)
        Eref = expm(X) - np.eye(len(X))
        assert np.abs(E - Eref).max() > 1e-6 * np.abs(Eref).max(), kw


@pytest.mark.parametrize("d", [0.3, 1e-2, 1e-4])
def test_newton_schulz_contracts_the_purity_error(d):
    """On a canonical form with singular values 1 + d_j, one iteration gives
    1 + d -> 1 - 1.5 d^2 - 0.5 d^3 (X (3 + X^2) / 2 with X^2 = -(1 + d)^2)."""
    rng = np.random.default_rng(21)
    n = 8
    ds_ = d * rng.uniform(-1.0, 1.0, n // 2)
    J = np.zeros((n, n))
    for j, dj in enumerate(ds_):
        J[2 * j, 2 * j + 1], J[2 * j + 1, 2 * j] = 1.0 + dj, -(1.0 + dj)
    O, _ = np.linalg.qr(rng.standard_normal((n, n)))
    X = O @ J @ O.T
    X = 0.5 * (X - X.T)
    out = _ns(X, X @ X)
    sv = np.sort(np.linalg.svd(out, compute_uv=False))
    want = np.sort(np.repeat(1.0 - 1.5 * ds_ ** 2 - 0.5 * ds_ ** 3, 2))
    assert np.abs(sv - want).max() < 1e-14
