"""The algebra of the blocked complex Pfaffian the CUDA path runs (CPU): a numpy
transcription of the panel's Parlett-Reid steps with pending rank-2 terms
(T, U), the symmetric interchange kept on the upper triangle only (two row
segments beyond p, the column segment of p between q and p, the sign of
Y[q][p]), and the trailing update that reads its C_in from the upper triangle,
C_in(r, c) = -Y[c][r], computes the lower entries and mirrors them; against
the oracle's Pfaffian.  A variant that keeps the full-matrix row swap without
the column part is caught."""
import numpy as np
import pytest

from oracle import sgs_oracle as orc


def panel_steps(Y, k0, bs, flip, pf, upper_swap=True):
    """bs elimination steps from column k0 on the upper triangle of Y (in place);
    returns (T, U, flip, pf) with T, U [bs][n]."""
    n = Y.shape[0]
    T = np.zeros((bs, n), complex)
    U = np.zeros((bs, n), complex)

    def column(k, lo, s):
        # column k below row lo - 1: -Y[k][i] (upper triangle) plus the pending terms
        v = np.zeros(n, complex)
        i = np.arange(lo, n)
        v[i] = -Y[k, i] + (T[:s, i] * U[:s, k][:, None] - U[:s, i] * T[:s, k][:, None]).sum(axis=0)
        return v

    for s in range(bs):
        k = k0 + 2 * s
        ck = column(k, k + 1, s)
        p = k + 1 + int(np.argmax(np.abs(ck[k + 1:])))
        q = k + 1
        if p != q:
            if upper_swap:
                for j in range(p + 1, n):
                    Y[q, j], Y[p, j] = Y[p, j], Y[q, j]
                for c in range(q + 1, p):
                    a = Y[q, c]
                    Y[q, c] = -Y[c, p]
                    Y[c, p] = -a
                Y[q, p] = -Y[q, p]
            else:                                  # a row swap alone: misses the column part
                Y[[q, p], k:] = Y[[p, q], k:]
            T[:s, [q, p]] = T[:s, [p, q]]
            U[:s, [q, p]] = U[:s, [p, q]]
            ck[[q, p]] = ck[[p, q]]
            flip ^= 1
        c1 = column(k + 1, k + 2, s)
        piv = -ck[k + 1]
        pf *= piv
        T[s, k + 2:] = -ck[k + 2:] / piv
        U[s, k + 2:] = c1[k + 2:]
    return T, U, flip, pf


def trailing_update(Y, e0, T, U):
    """Rows and columns e0 .. n - 1: C(r, c) = -Y[c][r] + sum_t (T_t[r] U_t[c] - U_t[r] T_t[c]) for
    r > c (C_in from the upper triangle, beta = -1), mirrored to Y[c][r] = -C(r, c); zero diagonal."""
    n = Y.shape[0]
    upd = T[:, e0:].T @ U[:, e0:] - U[:, e0:].T @ T[:, e0:]
    C = -Y[e0:, e0:].T + upd
    low = np.tril(np.ones((n - e0, n - e0), bool), -1)
    blk = np.where(low, C, 0.0)
    Y[e0:, e0:] = blk - blk.T


def blocked_pfaffian(Y, bs, upper_swap=True):
    Y = Y.copy()
    n = Y.shape[0]
    flip, pf = 0, 1.0 + 0.0j
    for k0 in range(0, n, 2 * bs):
        b = min(bs, (n - k0) // 2)
        T, U, flip, pf = panel_steps(Y, k0, b, flip, pf, upper_swap)
        e0 = k0 + 2 * b
        if e0 < n:
            trailing_update(Y, e0, T, U)
    return -pf if flip else pf


@pytest.mark.parametrize("n,bs", [(8, 2), (14, 3), (20, 4), (24, 5), (16, 8)])
def test_upper_triangle_pfaffian(n, bs):
    rng = np.random.default_rng(n + 7 * bs)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Y = X - X.T
    ref_phase, ref_log = orc.pfaffian_log(Y)
    pf = blocked_pfaffian(Y, bs)
    assert abs(np.log(abs(pf)) - ref_log) < 1e-11 * max(1.0, abs(ref_log))
    assert abs(pf / abs(pf) - ref_phase) < 1e-11
    # the lower triangle of the live part goes stale, so nothing else may read it: scrambling it
    # between panels changes nothing (the transcription reads only the upper triangle)
    Z = Y.copy()
    Z[np.tril_indices(n, -1)] = rng.standard_normal(n * (n - 1) // 2)
    pz = blocked_pfaffian(Z, bs)
    assert abs(pz - pf) <= 1e-12 * abs(pf)


def test_row_swap_alone_is_caught():
    """Interchanges that swap rows only, without the column segment and the sign of Y[q][p]
    that the upper triangle needs, give a wrong Pfaffian."""
    rng = np.random.default_rng(3)
    n = 16
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Y = X - X.T
    ref_phase, ref_log = orc.pfaffian_log(Y)
    bad = blocked_pfaffian(Y, 4, upper_swap=False)
    assert abs(np.log(abs(bad)) - ref_log) > 1e-6 or abs(bad / abs(bad) - ref_phase) > 1e-6


def test_update_packs_give_the_rank_2b_update():
    """The four packs the panel writes (as FP64 or as slices), with the source plane and sign of
    each block as the panel takes them (A_re: block src, negated for Ti and Ur; A_im: block src,
    negated for Ur and Ui; B_re: plane (blk + 2) & 3; B_im: plane 3 - blk; planes Tr, Ti, Ur, Ui),
    give Re and Im of T U^T - U T^T as A_re B_re^T and A_im B_im^T."""
    rng = np.random.default_rng(5)
    bs, n = 5, 11
    T = rng.standard_normal((bs, n)) + 1j * rng.standard_normal((bs, n))
    U = rng.standard_normal((bs, n)) + 1j * rng.standard_normal((bs, n))
    planes = [T.real, T.imag, U.real, U.imag]

    def pack(src_of, neg_of):
        return np.concatenate([(-1.0 if neg_of(b) else 1.0) * planes[src_of(b)].T for b in range(4)], axis=1)

    A_re = pack(lambda b: b, lambda b: b in (1, 2))
    A_im = pack(lambda b: b, lambda b: b >= 2)
    B_re = pack(lambda b: (b + 2) & 3, lambda b: False)
    B_im = pack(lambda b: 3 - b, lambda b: False)
    ref = T.T @ U - U.T @ T
    assert np.abs(A_re @ B_re.T - ref.real).max() < 1e-13
    assert np.abs(A_im @ B_im.T - ref.imag).max() < 1e-13
