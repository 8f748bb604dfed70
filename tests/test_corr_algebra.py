"""The spin correlator's closed form (Eq. Cr, Eq. K2CK) as the CUDA path
evaluates it, on the CPU, against the oracle's Wick expansion of the spin
operators' Majorana polynomials.

For sites 0 and s != 0 the kernel takes, per spin component a, the
antisymmetric 4 x 4 matrix K^a of S^a = (i/8) sum_pq K^a_pq c_p c_q and the
4 x 4 blocks B00, Bss, B0s of Delta:
  <S^a(0) S^a(s)> = [ (K:B00)(K:Bss) - 2 tr(K^T B0s K B0s^T) ] / 64,
and for s = 0, S(0).S(0) = 3/4 (n_up + n_dn - 2 n_up n_dn) with n_up =
(1 - D01)/2, n_dn = (1 - D23)/2 and n_up n_dn = (1 - D01 - D23 + Pf D[0:4])/4.
Both are identities of Wick's theorem, so they hold for any complex
antisymmetric Delta, transition matrices included.  Planted mistakes (the
relative sign of K^y's two entries, the trace term's factor 2) are caught; the
overall sign of a K^a cannot matter, since each term is quadratic in it."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc


def kspin(a, flip_y=False):
    K = np.zeros((4, 4))
    if a == 2:
        K[0, 1], K[2, 3] = 1.0, -1.0
    elif a == 0:
        K[0, 3], K[1, 2] = 1.0, -1.0
    else:
        K[0, 2], K[1, 3] = (-1.0, 1.0) if flip_y else (-1.0, -1.0)
    return K - K.T


def spin_dot_value(D, s, flip_y=False, trace_factor=2.0):
    if s == 0:
        d01, d23 = D[0, 1], D[2, 3]
        pf = D[0, 1] * D[2, 3] - D[0, 2] * D[1, 3] + D[0, 3] * D[1, 2]
        nu, nv = 0.5 * (1 - d01), 0.5 * (1 - d23)
        nn = 0.25 * (1 - d01 - d23 + pf)
        return 0.75 * (nu + nv - 2 * nn)
    B00 = D[0:4, 0:4]
    Bss = D[4 * s:4 * s + 4, 4 * s:4 * s + 4]
    B0s = D[0:4, 4 * s:4 * s + 4]
    tot = 0.0
    for a in range(3):
        K = kspin(a, flip_y)
        k0 = (K * B00).sum()
        ks = (K * Bss).sum()
        tr = np.trace(K.T @ B0s @ K @ B0s.T)
        tot += (k0 * ks - trace_factor * tr) / 64.0
    return tot


def _random_antisym(n, rng):
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return X - X.T


@pytest.mark.parametrize("s", [0, 1, 2, 5])
def test_closed_form_equals_the_wick_expansion(s):
    rng = np.random.default_rng(s + 3)
    n = 4 * 6
    for D in (_random_antisym(n, rng), inp.random_pure_gamma(n // 2, rng).astype(complex)):
        ref = orc.poly_expectation(orc.spin_dot(0, s), D)
        got = spin_dot_value(D, s)
        assert abs(got - ref) < 1e-12 * max(1.0, abs(ref))


def test_on_transition_matrices():
    rng = np.random.default_rng(9)
    N = 12
    Ga, Gb = inp.random_pure_gamma(N, rng), inp.random_pure_gamma(N, rng)
    D = orc.transition_matrix(Gb, Ga)            # Delta^{b,a}, as the kernel reads it
    for s in range(N // 2):
        ref = orc.poly_expectation(orc.spin_dot(0, s), D)
        assert abs(spin_dot_value(D, s) - ref) < 1e-12 * max(1.0, abs(ref))


def test_singlet_value_on_the_impurity():
    """A singly occupied site has S(0).S(0) = 3/4; empty and doubly occupied sites 0."""
    N = 2
    J = inp.vacuum_gamma(N).astype(complex)      # both modes empty
    assert abs(spin_dot_value(J, 0)) < 1e-15
    one = J.copy()
    one[0:2, 0:2] *= -1.0                        # the up mode occupied
    assert abs(spin_dot_value(one, 0) - 0.75) < 1e-15
    two = -J                                     # both occupied
    assert abs(spin_dot_value(two, 0)) < 1e-15


def test_planted_mistakes_are_caught():
    rng = np.random.default_rng(4)
    D = _random_antisym(16, rng)
    ref = orc.poly_expectation(orc.spin_dot(0, 2), D)
    assert abs(spin_dot_value(D, 2, flip_y=True) - ref) > 1e-6 * abs(ref)
    assert abs(spin_dot_value(D, 2, trace_factor=1.0) - ref) > 1e-6 * abs(ref)
