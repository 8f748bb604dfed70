"""The lower-tile scheme the assembly kernels share (pair Q, the equation of
motion's two passes), on the CPU: block t of a launch of lower_tile_count(n)
blocks takes tile (K, L) = lower_tile(t), K >= L, of 32 x 32, computes the
entries strictly below the diagonal and stores them with their mirror
(store_antisym_tile): tile (K, L) directly, tile (L, K) as -s^T, and on a
diagonal tile the upper part as the negated transpose and a zero diagonal.
An optional mask keeps entries the block did not compute.  The transcription
must rebuild any antisymmetric matrix exactly, ragged edges included, from
tiles whose upper and diagonal entries hold garbage.  Also the Renyi kernels'
decode of a block index into a pair of pairs (u <= v)."""
import numpy as np
import pytest


def lower_tile_count(n):
    t = (n + 31) // 32
    return t * (t + 1) // 2


def lower_tile(t):
    k = 0
    while (k + 1) * (k + 2) // 2 <= t:
        k += 1
    return k, t - k * (k + 1) // 2


def store_antisym_tile(x, n, k0, l0, s, have=None):
    for j in range(32):
        for tx in range(32):
            k, l = k0 + j, l0 + tx
            if k < n and l < n:
                if k0 != l0:
                    if have is None or have[j][tx]:
                        x[k, l] = s[j][tx]
                elif k > l:
                    if have is None or have[j][tx]:
                        x[k, l] = s[j][tx]
                elif k < l:
                    if have is None or have[tx][j]:
                        x[k, l] = -s[tx][j]
                else:
                    if have is None or have[j][tx]:
                        x[k, l] = 0.0
            if k0 != l0:
                r, c = l0 + j, k0 + tx
                if r < n and c < n and (have is None or have[tx][j]):
                    x[r, c] = -s[tx][j]


def assemble(src, n, rng, mask=None, init=None):
    """Every block of the launch: its tile of src's strictly lower entries (garbage elsewhere),
    stored with its mirror; mask[k, l] (k > l) marks the entries computed."""
    x = np.full((n, n), np.nan) if init is None else init.copy()
    for t in range(lower_tile_count(n)):
        K, L = lower_tile(t)
        k0, l0 = 32 * K, 32 * L
        s = rng.standard_normal((32, 33))                       # garbage where nothing is computed
        have = np.zeros((32, 33), bool) if mask is not None else None
        for j in range(32):
            for c in range(32):
                k, l = k0 + j, l0 + c
                if k < n and l < n and k > l and (mask is None or mask[k, l]):
                    s[j][c] = src[k, l]
                    if have is not None:
                        have[j][c] = True
        store_antisym_tile(x, n, k0, l0, s, have)
    return x


def test_tiles_cover_the_lower_triangle_once():
    for n in (1, 31, 32, 33, 64, 65, 200, 512):
        T = (n + 31) // 32
        tiles = [lower_tile(t) for t in range(lower_tile_count(n))]
        assert sorted(tiles) == sorted((K, L) for K in range(T) for L in range(K + 1))


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 70, 96])
def test_store_rebuilds_the_antisymmetric_matrix(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n))
    A = X - X.T
    got = assemble(A, n, rng)
    assert np.array_equal(got, A)


def test_masked_store_keeps_what_was_not_computed():
    """The impurity-terms pass of the equation of motion computes only rows and columns of
    the interacting modes: with a mask, every other entry keeps its value."""
    rng = np.random.default_rng(5)
    n = 70
    X = rng.standard_normal((n, n))
    A = X - X.T
    Y = rng.standard_normal((n, n))
    before = Y - Y.T
    imp = [0, 1, 33, 65]
    mask = np.zeros((n, n), bool)
    mask[imp, :] = True
    mask[:, imp] = True
    got = assemble(A, n, rng, mask=mask, init=before)
    want = np.where(mask, A, before)                # both zero on the diagonal
    assert np.array_equal(got, want)


def decode_pair_of_pairs(q):
    """The Renyi kernels' decode of a block index q = v (v + 1) / 2 + u, u <= v: a double
    square root, then integer corrections in both directions."""
    import math
    v = int((math.sqrt(8.0 * float(q) + 1.0) - 1.0) * 0.5)
    while (v + 1) * (v + 2) // 2 <= q:
        v += 1
    while v * (v + 1) // 2 > q:
        v -= 1
    return q - v * (v + 1) // 2, v


def test_pair_of_pairs_decode_is_exact():
    """Every q of a launch maps to one (u, v) with u <= v, in order, including indices far past
    any rank the library admits (where the square root's rounding needs the corrections)."""
    q = 0
    for v in range(300):
        for u in range(v + 1):
            assert decode_pair_of_pairs(q) == (u, v)
            q += 1
    rng = np.random.default_rng(2)
    for v in list(rng.integers(1, 2 ** 26, 2000)) + [2 ** 26 - 1, 94906265, 94906266]:
        v = int(v)
        for u in (0, v // 2, v):
            assert decode_pair_of_pairs(v * (v + 1) // 2 + u) == (u, v)
