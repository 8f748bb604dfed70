"""The algebra of the Gauss-Jordan inverse the CUDA path runs (CPU): a numpy
transcription of the panel kernel's in-place elimination with partial
pivoting, of the delayed update (pivot rows replaced, other rows added to),
and of the recursive order (left half, its update of the right half's
columns, right half, its update of the left half's columns), against numpy's
inverse and determinant and against the one-level blocked order."""
import numpy as np
import pytest


def panel(W, k0, bb, piv, logdet):
    """Eliminate columns k0 .. k0 + bb - 1 in place (gj_panel_kernel): the panel's
    interchanges go to every other column, its pivot rows (other columns) are returned
    as the update operand."""
    n = W.shape[0]
    P = W[:, k0:k0 + bb].copy()
    for j in range(bb):
        c = k0 + j
        p = c + int(np.argmax(np.abs(P[c:, j])))
        P[[c, p]] = P[[p, c]]
        piv[c] = p
        inv = 1.0 / P[c, j]
        logdet[0] += np.log(abs(P[c, j]))
        rowc = P[c] * inv
        rowc[j] = inv
        P[c] = rowc
        for r in range(n):
            if r == c:
                continue
            f = P[r, j]
            for q in range(bb):
                if q != j:
                    P[r, q] -= f * rowc[q]
            P[r, j] = -f * inv
    W[:, k0:k0 + bb] = P
    other = np.r_[0:k0, k0 + bb:n]
    for j in range(bb):
        c, p = k0 + j, piv[k0 + j]
        if p != c:
            W[np.ix_([c, p], other)] = W[np.ix_([p, c], other)]


def update(W, p0, K, t0, w):
    """Target columns t0 .. t0 + w - 1 by the eliminated columns p0 .. p0 + K - 1
    (gj_update): pivot rows replaced, the other rows added to."""
    T = W[p0:p0 + K, t0:t0 + w].copy()
    prod = W[:, p0:p0 + K] @ T
    tgt = W[:, t0:t0 + w]
    keep = np.ones(W.shape[0], bool)
    keep[p0:p0 + K] = False
    W[:, t0:t0 + w] = prod + np.where(keep[:, None], tgt, 0.0)


def recurse(W, c0, c1, leaf, piv, logdet):
    if c1 - c0 <= leaf:
        panel(W, c0, c1 - c0, piv, logdet)
        return
    leaves = -(-(c1 - c0) // leaf)
    m = c0 + ((leaves + 1) // 2) * leaf
    recurse(W, c0, m, leaf, piv, logdet)
    update(W, c0, m - c0, m, c1 - m)
    recurse(W, m, c1, leaf, piv, logdet)
    update(W, m, c1 - m, c0, m - c0)


def flat(W, leaf, piv, logdet):
    n = W.shape[0]
    for k0 in range(0, n, leaf):
        bb = min(leaf, n - k0)
        panel(W, k0, bb, piv, logdet)
        # every other column at once
        T = W[k0:k0 + bb].copy()
        T[:, k0:k0 + bb] = 0.0
        prod = W[:, k0:k0 + bb] @ T
        keep = np.ones(n, bool)
        keep[k0:k0 + bb] = False
        cols = np.r_[0:k0, k0 + bb:n]
        W[:, cols] = (prod + np.where(keep[:, None], W, 0.0))[:, cols]


def unpermute(W, piv):
    n = W.shape[0]
    pm = list(range(n))
    for j in range(n - 1, -1, -1):
        p = piv[j]
        if p != j:
            pm[j], pm[p] = pm[p], pm[j]
    return W[:, pm]


@pytest.mark.parametrize("n,leaf", [(20, 4), (37, 8), (64, 8), (64, 16), (50, 24)])
def test_recursive_inverse(n, leaf):
    rng = np.random.default_rng(n + leaf)
    X = rng.standard_normal((n, n))
    S = X - X.T if n % 2 == 0 else X + n ** 0.5 * np.eye(n)
    W = S.copy()
    piv = np.zeros(n, int)
    ld = np.zeros(1)
    recurse(W, 0, n, leaf, piv, ld)
    inv = unpermute(W, piv)
    ref = np.linalg.inv(S)
    assert np.abs(inv - ref).max() <= 1e-11 * np.abs(ref).max()
    assert abs(ld[0] - np.linalg.slogdet(S)[1]) <= 1e-11 * max(1.0, abs(ld[0]))
    # the one-level blocked order gives the same pivots and the same inverse to rounding
    W2 = S.copy()
    piv2 = np.zeros(n, int)
    flat(W2, leaf, piv2, np.zeros(1))
    assert np.array_equal(piv, piv2)
    assert np.abs(unpermute(W2, piv2) - inv).max() <= 1e-11 * np.abs(ref).max()


def test_dropping_the_second_update_is_caught():
    """A recursion that forgets to update the left half by the right half is wrong."""
    n, leaf = 24, 4
    rng = np.random.default_rng(0)
    X = rng.standard_normal((n, n))
    S = X - X.T
    W = S.copy()
    piv = np.zeros(n, int)

    def broken(W, c0, c1):
        if c1 - c0 <= leaf:
            panel(W, c0, c1 - c0, piv, np.zeros(1))
            return
        m = c0 + ((-(-(c1 - c0) // leaf) + 1) // 2) * leaf
        broken(W, c0, m)
        update(W, c0, m - c0, m, c1 - m)
        broken(W, m, c1)

    broken(W, 0, n)
    assert np.abs(unpermute(W, piv) - np.linalg.inv(S)).max() > 1e-3


def update_chunked(W, p0, K, t0, w, kc):
    """update() in K chunks of kc (the emulated product's chunks of 512): the first chunk replaces
    the pivot rows like update(), the later ones add onto every row (gj_acc)."""
    T = W[p0:p0 + K, t0:t0 + w].copy()
    keep = np.ones(W.shape[0], bool)
    keep[p0:p0 + K] = False
    out = None
    for c0 in range(0, K, kc):
        c1 = min(K, c0 + kc)
        prod = W[:, p0 + c0:p0 + c1] @ T[c0:c1]
        if out is None:
            out = prod + np.where(keep[:, None], W[:, t0:t0 + w], 0.0)
        else:
            out = out + prod
    W[:, t0:t0 + w] = out


@pytest.mark.parametrize("K,kc", [(10, 4), (12, 12), (13, 5)])
def test_k_chunked_update_equals_one_update(K, kc):
    rng = np.random.default_rng(K + kc)
    n, p0, t0, w = 40, 6, 25, 9
    W = rng.standard_normal((n, n))
    a, b = W.copy(), W.copy()
    update(a, p0, K, t0, w)
    update_chunked(b, p0, K, t0, w, kc)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    # a later chunk that replaced the pivot rows again would drop the first chunk's product
    if kc < K:
        c = W.copy()
        T = c[p0:p0 + K, t0:t0 + w].copy()
        keep = np.ones(n, bool)
        keep[p0:p0 + K] = False
        out = c[:, p0:p0 + kc] @ T[:kc] + np.where(keep[:, None], c[:, t0:t0 + w], 0.0)
        out2 = c[:, p0 + kc:p0 + K] @ T[kc:] + np.where(keep[:, None], out, 0.0)
        c[:, t0:t0 + w] = out2
        assert np.abs(c - a).max() > 1e-6
