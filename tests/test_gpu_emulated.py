"""FP64 products emulated on the bf16 tensor cores (the library's default
FP64 arithmetic) (GPU).

Error of one emulated product C = alpha op(A) op(B) + beta Cin + diag I, per
element, against a reference in extended precision (numpy longdouble: at
least 64 significand bits), u = 2^-53:

    |C_ij - ref_ij| <= |alpha| K 2^-52 max_k |A_ik| max_k |B_kj|
                       + (4 + c) u (|alpha| (|A||B|)_ij + |beta Cin_ij| + |diag|)

with c the number of K chunks of 512.  The first term is the slicing: every
K-major row of op(A) and column of op(B) keeps 57 fractional bits of its
largest entry's power of two (2^-56 of the row's maximum per entry) and the
slice products of combined weight below 2^-63 are dropped (at most 2^-53.2 of
the two maxima per term); the fp32 group sums above 2^24 (K > 455) add at most
2^-48 of the maxima.  So a row whose entries are far below its largest keeps
fewer bits than an FP64 product would, and the bound is normwise per row and
column, not elementwise: test_uneven_rows_hit_the_normwise_bound shows a case
where the error exceeds the elementwise FP64 bound by orders and stays within
this one.  The second term covers the FP64 roundings of the combination and
the epilogue.  The arithmetic of the scheme is pinned in exact rational
arithmetic on the CPU (tests/test_emulation_scheme.py).  The factorisations
and whole steps built on it are held to the FP64 bars (the oracle at 1e-10)."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu
U = 2.0 ** -53
EMU = 0
KC = 512


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def _operands(rng, batch, m, n, k, trans_a, trans_b):
    A = rng.standard_normal((batch, m, k)) * 10.0 ** rng.uniform(-3, 3, (batch, m, 1))
    B = rng.standard_normal((batch, k, n)) * 10.0 ** rng.uniform(-3, 3, (batch, 1, n))
    A[:, m // 2] = 0.0                                    # a zero row
    if k > 3:
        A[:, 0, 1] *= 1e-9                                # a row of uneven magnitudes
    As = np.swapaxes(A, 1, 2).copy() if trans_a else A
    Bs = np.swapaxes(B, 1, 2).copy() if trans_b else B
    return A, B, As, Bs


def _exact(A, B):
    return np.matmul(A.astype(np.longdouble), B.astype(np.longdouble))


def emulated_bound(A, B, alpha=1.0, Cin=None, beta=0.0, diag=0.0):
    """The error bound of the module docstring, elementwise, for op(A) = A, op(B) = B."""
    k = A.shape[-1]
    chunks = -(-k // KC)
    ra = np.abs(A).max(axis=-1, keepdims=True)
    cb = np.abs(B).max(axis=-2, keepdims=True)
    m, n = A.shape[-2], B.shape[-1]
    add = abs(alpha) * (np.abs(A) @ np.abs(B)) + abs(diag) * np.eye(m, n)
    if Cin is not None:
        add = add + abs(beta) * np.abs(Cin)
    return abs(alpha) * k * 2.0 ** -52 * ra * cb + (4 + chunks) * U * add


def _err(C, ref):
    return np.abs(C.astype(np.longdouble) - ref).astype(np.float64)


SHAPES = [
    (1, 1, 1, 1, False, False),
    (2, 128, 64, 64, False, False),
    (2, 300, 200, 104, False, True),       # ragged tiles, K tail
    (3, 130, 70, 33, True, False),
    (1, 96, 80, 300, True, True),
    (2, 64, 64, 512, False, False),        # one full K chunk
    (1, 96, 80, 804, False, True),         # K in two chunks
    (3, 512, 16, 16, False, False),        # 128 x 16 tiles (n <= 16): a Gauss-Jordan leaf update's shape
    (2, 300, 7, 40, True, True),           # 128 x 16 tiles, ragged rows and columns
]


@pytest.mark.parametrize("batch,m,n,k,ta,tb", SHAPES)
def test_product_matches_extended_reference(pkg, batch, m, n, k, ta, tb):
    rng = np.random.default_rng(m * 7 + n + k)
    A, B, As, Bs = _operands(rng, batch, m, n, k, ta, tb)
    C = pkg.batched_gemm(As, Bs, trans_a=ta, trans_b=tb, fp64_path=EMU)
    ref = _exact(A, B)
    bound = emulated_bound(A, B)
    err = _err(C, ref)
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()
    assert np.all(C[:, m // 2] == 0.0)


@pytest.mark.parametrize("k", [2, 40, 512, 804])
def test_uneven_rows_hit_the_normwise_bound(pkg, k):
    """Rows with one large entry and the rest 1e-9 .. 1e-12 of it, against columns
    that are zero where the row is large: the exact result is made of the small
    entries alone.  The emulated product keeps only 57 bits of the row's largest
    entry's scale for them, so its error exceeds the elementwise bound
    4 u (|A||B|) of an FP64 product by orders; the normwise bound holds."""
    rng = np.random.default_rng(k)
    batch, m, n = 2, 130, 70
    A = rng.standard_normal((batch, m, k)) * 10.0 ** rng.uniform(-12, -9, (batch, m, k))
    A[:, :, 0] = rng.choice([-1.0, 1.0], (batch, m)) * rng.uniform(1.0, 2.0, (batch, m))
    B = rng.standard_normal((batch, k, n))
    B[:, 0, :] = 0.0
    B[:, 0, ::7] = rng.standard_normal((batch, (n + 6) // 7))       # some columns see the large entry
    C = pkg.batched_gemm(A, B, fp64_path=EMU)
    ref = _exact(A, B)
    err = _err(C, ref)
    bound = emulated_bound(A, B)
    assert np.all(err <= bound), (err / bound).max()
    elementwise = 4 * U * (np.abs(A) @ np.abs(B))
    assert (err / elementwise).max() > 1e3           # the case is what it claims
    # the FP64 FMA path meets the elementwise bound on the same operands
    Cf = pkg.batched_gemm(A, B, fp64_path=1)
    assert np.all(_err(Cf, ref) <= k * U * (np.abs(A) @ np.abs(B)))


def test_epilogue_terms_and_batch_chunks(pkg):
    """alpha, beta Cin, diag on a square product; a small scratch forces the
    batch into chunks without changing a bit of the result."""
    rng = np.random.default_rng(5)
    batch, n, k = 5, 160, 96
    A = rng.standard_normal((batch, n, k))
    B = rng.standard_normal((batch, k, n))
    Cin = rng.standard_normal((batch, n, n))
    C1 = pkg.batched_gemm(A, B, Cin=Cin, alpha=-0.37, beta=1.5, diag=0.25, fp64_path=EMU)
    ref = -0.37 * _exact(A, B) + 1.5 * Cin.astype(np.longdouble) + 0.25 * np.eye(n)
    bound = emulated_bound(A, B, -0.37, Cin, 1.5, 0.25)
    assert np.all(_err(C1, ref) <= bound)
    C2 = pkg.batched_gemm(A, B, Cin=Cin, alpha=-0.37, beta=1.5, diag=0.25, fp64_path=EMU,
                          emulation_scratch=3 << 20)      # about one batch entry per chunk
    assert np.array_equal(C1, C2)


EPILOGUES = [(1.0, None, 0.0), (1.0, None, 0.5), (-0.5, None, 0.0), (1.0, 1.0, 0.0), (1.0, 1.0, 0.5),
             (-0.5, 1.0, 0.25), (4.0, 0.75, 0.0), (3.0, 1.0, -1.5)]


@pytest.mark.parametrize("alpha,beta,diag", EPILOGUES)
def test_epilogue_forms(pkg, alpha, beta, diag):
    """Each form of the store pass (the plain product, the in-place update C = Cin + A B,
    the general one), with alpha a power of two or not and with and without the diagonal
    term, on ragged tiles of a rectangular product."""
    rng = np.random.default_rng(int(abs(alpha) * 100 + (beta or 0) * 10 + diag * 4 + 50))
    batch, m, n, k = 2, 150, 100, 40
    A = rng.standard_normal((batch, m, k))
    B = rng.standard_normal((batch, k, n))
    Cin = None if beta is None else rng.standard_normal((batch, m, n))
    C = pkg.batched_gemm(A, B, Cin=Cin, alpha=alpha, beta=beta or 0.0, diag=diag, fp64_path=EMU)
    ref = alpha * _exact(A, B) + diag * np.eye(m, n)
    if Cin is not None:
        ref = ref + beta * Cin.astype(np.longdouble)
    bound = emulated_bound(A, B, alpha, Cin, beta or 0.0, diag)
    err = _err(C, ref)
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()


@pytest.mark.parametrize("scale", [1e-158, 1e158])
def test_results_below_and_beyond_the_normal_range(pkg, scale):
    """Products of magnitude near 1e-316 come out on the subnormal grid (within one of its
    units), those near 1e316 as infinities of the right sign; elements that cancel back into
    the normal range keep the usual bound."""
    rng = np.random.default_rng(21)
    batch, m, n, k = 2, 130, 70, 40
    A = rng.standard_normal((batch, m, k)) * scale
    B = rng.standard_normal((batch, k, n)) * scale
    C = pkg.batched_gemm(A, B, fp64_path=EMU)
    ref = _exact(A, B)
    if scale < 1:
        bound = emulated_bound(A, B) + 2.0 ** -1074
        err = _err(C, ref)
        assert np.all(err <= bound), (err / bound).max()
        assert np.all(np.abs(C) < 2.2250738585072014e-308)
    else:
        big = np.abs(ref) > np.longdouble("1e309")
        assert big.mean() > 0.9
        with np.errstate(over="ignore"):
            sign = np.sign(ref[big].astype(np.float64))
        assert np.all(np.isinf(C[big])) and np.all(np.sign(C[big]) == sign)
        small = np.abs(ref) < np.longdouble("1e307")
        Al, Bl = A.astype(np.longdouble), B.astype(np.longdouble)
        bound = (40 * 2.0 ** -52 * np.abs(Al).max(axis=-1, keepdims=True) * np.abs(Bl).max(axis=-2, keepdims=True)
                 + 5 * U * (np.abs(Al) @ np.abs(Bl)))
        assert np.all(np.abs(C[small].astype(np.longdouble) - ref[small]) <= bound[small])


def test_antisymmetric_mode(pkg):
    rng = np.random.default_rng(9)
    batch, n = 2, 200
    G = rng.standard_normal((batch, n, n))
    G = G - np.swapaxes(G, 1, 2)
    S = rng.standard_normal((batch, n, n))
    S = S - np.swapaxes(S, 1, 2)
    # G S G is antisymmetric for antisymmetric G and S: A = G S, B = G
    A = np.matmul(G, S)
    Cin = rng.standard_normal((batch, n, n))
    Cin = Cin - np.swapaxes(Cin, 1, 2)
    C = pkg.batched_gemm(A, G, Cin=Cin, beta=0.5, mode=1, fp64_path=EMU)
    ref = _exact(A, G) + 0.5 * Cin.astype(np.longdouble)
    low = np.tril(np.ones((n, n), dtype=bool), -1)
    bound = emulated_bound(A, G, 1.0, Cin, 0.5)
    err = _err(C, ref)
    assert np.all(err[:, low] <= bound[:, low])
    assert np.array_equal(C, -np.swapaxes(C, 1, 2))
    assert np.all(np.diagonal(C, axis1=1, axis2=2) == 0.0)
    # without Cin (the plain product's store pass)
    C0 = pkg.batched_gemm(A, G, mode=1, fp64_path=EMU)
    err0 = _err(C0, _exact(A, G))
    assert np.all(err0[:, low] <= emulated_bound(A, G)[:, low])
    assert np.array_equal(C0, -np.swapaxes(C0, 1, 2))
    assert np.all(np.diagonal(C0, axis1=1, axis2=2) == 0.0)


@pytest.mark.parametrize("n,mode,alpha", [(200, 0, 0.7), (200, 1, -0.5), (600, 0, 1.0), (600, 1, 0.3)])
def test_antisymmetric_b_sliced_by_rows(pkg, n, mode, alpha):
    """B declared antisymmetric: its rows are sliced in place of op(B)'s columns and alpha
    changes sign; K = 600 runs in two chunks (the K range taken within B's rows)."""
    rng = np.random.default_rng(n + 10 * mode)
    batch = 2
    G = rng.standard_normal((batch, n, n))
    G = G - np.swapaxes(G, 1, 2)
    S = rng.standard_normal((batch, n, n))
    S = S - np.swapaxes(S, 1, 2)
    A = np.matmul(G, S) if mode == 1 else rng.standard_normal((batch, n, n))
    C = pkg.batched_gemm(A, G, alpha=alpha, mode=mode, b_antisym=True, fp64_path=EMU)
    ref = alpha * _exact(A, G)
    bound = emulated_bound(A, G, alpha)
    err = _err(C, ref)
    sel = np.tril(np.ones((n, n), dtype=bool), -1) if mode == 1 else np.ones((n, n), dtype=bool)
    assert np.all(err[:, sel] <= bound[:, sel]), (err / np.maximum(bound, 1e-300))[:, sel].max()
    if mode == 1:
        assert np.array_equal(C, -np.swapaxes(C, 1, 2))


def test_narrow_tiles_antisymmetric_mode(pkg):
    """Products of at most 16 output columns run on 128 x 16 tiles (SHAPES has two plain ones):
    a 16 x 16 antisymmetric product, lower tiles computed and mirrored.  The Gauss-Jordan
    updates of 16 target columns take the same tiles inside every inverse of n >= 32
    (test_inverse_emulated, the step tests)."""
    rng = np.random.default_rng(12)
    batch = 3
    G = rng.standard_normal((batch, 16, 16))
    G = G - np.swapaxes(G, 1, 2)
    S = rng.standard_normal((batch, 16, 16))
    S = S - np.swapaxes(S, 1, 2)
    A = np.matmul(G, S)
    C = pkg.batched_gemm(A, G, mode=1, fp64_path=EMU)
    low = np.tril(np.ones((16, 16), dtype=bool), -1)
    assert np.all(_err(C, _exact(A, G))[:, low] <= emulated_bound(A, G)[:, low])
    assert np.array_equal(C, -np.swapaxes(C, 1, 2))


@pytest.mark.parametrize("n,k0,b", [(192, 64, 32), (700, 50, 600)])
def test_gauss_jordan_mode_matches_native_semantics(pkg, n, k0, b):
    """Columns of the panel stay as they were; rows of the panel start from 0.  K = 600 runs
    as two K chunks: the second adds onto the pivot rows the first replaced."""
    rng = np.random.default_rng(11 + b)
    batch = 2
    A = rng.standard_normal((batch, n, b))
    B = rng.standard_normal((batch, b, n))
    W = rng.standard_normal((batch, n, n))
    C = pkg.batched_gemm(A, B, Cin=W, beta=1.0, mode=2, gj=(k0, b), C=W, fp64_path=EMU)
    Cn = pkg.batched_gemm(A, B, Cin=W, beta=1.0, mode=2, gj=(k0, b), C=W, fp64_path=1)
    cols = np.arange(n)
    panel = (cols >= k0) & (cols < k0 + b)
    assert np.array_equal(C[:, :, panel], W[:, :, panel])
    ref = _exact(A, B) + W.astype(np.longdouble)
    ref[:, k0:k0 + b, :] -= W[:, k0:k0 + b, :]
    bound = emulated_bound(A, B, 1.0, W, 1.0)
    err = _err(C, ref)
    assert np.all(err[:, :, ~panel] <= bound[:, :, ~panel])
    # the native product is within its own K-term bound of the same value
    base = (np.abs(A) @ np.abs(B)) + np.abs(W)
    assert np.all(np.abs(Cn - ref.astype(np.float64))[:, :, ~panel] <= (4 + b) * U * base[:, :, ~panel])


@pytest.mark.parametrize("n,batch", [(12, 3), (84, 2), (200, 1), (512, 2)])
def test_inverse_emulated(pkg, n, batch):
    rng = np.random.default_rng(300 + n)
    X = rng.standard_normal((batch, n, n))
    S = X - np.swapaxes(X, 1, 2)
    inv, ld = pkg.batched_inverse(S, fp64_path=EMU)
    for b in range(batch):
        ref = np.linalg.inv(S[b])
        assert np.abs(inv[b] - ref).max() < 1e-9 * np.abs(ref).max()
        assert abs(ld[b] - np.linalg.slogdet(S[b])[1]) < 1e-10 * max(1.0, abs(ld[b]))


@pytest.mark.parametrize("n,batch", [(6, 3), (66, 2), (256, 1)])
def test_pfaffian_emulated(pkg, n, batch):
    rng = np.random.default_rng(400 + n)
    Y = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    Y = Y - np.swapaxes(Y, 1, 2)
    ph, la = pkg.batched_pfaffian(Y, fp64_path=EMU)
    for b in range(batch):
        rph, rla = orc.pfaffian_log(Y[b])
        assert abs(la[b] - rla) < 1e-10 * max(1.0, abs(rla))
        assert abs(ph[b] - rph) < 1e-10


def test_trajectory_and_mixed_form(pkg):
    """20 steps of the small workload on the emulated path against the oracle,
    and the TF32 form with emulated FP64 products against the TF32 form with
    FMA ones (same tensor-core products: agreement to FP64 rounding growth).
    One step of either arithmetic against the oracle is in test_gpu_step.py."""
    w = inp.SMALL
    p = w.model
    g, lam = inp.initial_state(p.n_modes, w.rank, w.seed, w.parity)
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    s = pkg.Solver(m, g, lam, dtau=w.dtau, fp64_path=EMU)
    Eg = s.step(20)[0]
    s.close()
    Eo, _, _ = orc.run(orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V), list(g), w.dtau, 20)
    assert np.abs(Eg - Eo).max() <= 1e-10 * np.abs(Eo).max()
    q = inp.AndersonParams(n_bath=40, U=4.0, eps_d=-2.0, V=0.5)
    rng = np.random.default_rng(3)
    gq = inp.clustered_pure_gammas(q.n_modes, 5, rng, 1, spread=1.0)
    mq = pkg.build_anderson(q.n_bath, q.U, q.eps_d, q.V)
    out = []
    for path in (pkg.FP64_EMULATED, pkg.FP64_FMA):
        s = pkg.Solver(mq, gq, None, precision=1, fp64_path=path)
        out.append(s.step(3)[0])
        s.close()
    assert np.abs(out[0] - out[1]).max() <= 1e-9 * np.abs(out[1]).max()


@pytest.mark.parametrize("M,cap", [(5, 3 << 19), (9, 600 << 10)])
def test_panel_written_slices_equal_the_slicers(pkg, M, cap):
    """The Pfaffian panel writes the slices of its trailing update, and one kernel writes both
    operands' slices of a Gauss-Jordan update of K, w <= 64, when the whole batch fits the
    slice scratch; with a scratch too small for that the updates take their FP64 operands
    through the slicing kernels in batch chunks.  Both take the same digits and
    exponents, so G, h, dGamma and the energy agree to the bit.  n = 84: M = 5 has 6 phase
    Pfaffians (12 update entries, 2.4 MB, beyond 1.5 MiB); M = 9 has 28 (56 entries) and
    halves of 18 pairs whose leaf updates (50 KB an entry) exceed 600 KiB, while one entry of
    every product (at most 361 KB) fits both caps."""
    p = inp.AndersonParams(n_bath=20, U=3.0, eps_d=-1.5, V=0.7)
    rng = np.random.default_rng(41)
    g = inp.clustered_pure_gammas(p.n_modes, M, rng, 1, spread=1.0)
    lam = inp.random_amplitudes(M, rng)
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    out = []
    for cap in (0, cap):
        s = pkg.Solver(m, g, lam, dtau=0.05, fp64_path=EMU, emulation_scratch=cap)
        E = s.step(2)[0]
        Gg, hg = s.pair_matrices()
        out.append((E, Gg, hg, s.derivative()))
        s.close()
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)
