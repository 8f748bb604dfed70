"""FP64 products emulated on the bf16 tensor cores (FP64 path 2) (GPU).

Bar for one product: |C - (alpha AB + beta Cin + diag I)| <= 4 u (|alpha| |A||B| + |beta Cin| + |diag|)
elementwise, u = 2^-53, against a reference in extended precision (numpy
longdouble: at least 64 significand bits).  A native FP64 product of K terms
is bounded by K u |A||B|; the emulation keeps 57 bits of every operand row and
sums its integer slice products exactly, so 4 u holds with margin at any K.
The factorisations and whole steps built on it are held to the FP64 path's
own bars (the oracle at 1e-10)."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture()
def pkg():
    import os

    import paper_2105_01088_gb300 as p
    p.set_fp64_gemm_path(p.FP64_EMULATED)
    try:
        yield p
    finally:
        p.set_fp64_gemm_path(int(os.environ.get("SGS_FP64_GEMM_PATH", p.FP64_FMA)))
        p.set_emulation_scratch(2 << 30)


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


SHAPES = [
    (1, 1, 1, 1, False, False),
    (2, 128, 64, 64, False, False),
    (2, 300, 200, 104, False, True),       # ragged tiles, K tail
    (3, 130, 70, 33, True, False),
    (1, 96, 80, 300, True, True),
    (2, 64, 64, 512, False, False),        # one full K chunk
    (1, 96, 80, 804, False, True),         # K in two chunks
]


@pytest.mark.parametrize("batch,m,n,k,ta,tb", SHAPES)
def test_product_matches_extended_reference(pkg, batch, m, n, k, ta, tb):
    rng = np.random.default_rng(m * 7 + n + k)
    A, B, As, Bs = _operands(rng, batch, m, n, k, ta, tb)
    C = pkg.batched_gemm(As, Bs, trans_a=ta, trans_b=tb)
    ref = _exact(A, B)
    bound = 4 * U * (np.abs(A) @ np.abs(B))
    err = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()
    assert np.all(C[:, m // 2] == 0.0)


def test_epilogue_terms_and_batch_chunks(pkg):
    """alpha, beta Cin, diag on a square product; a small scratch forces the
    batch into chunks without changing a bit of the result."""
    rng = np.random.default_rng(5)
    batch, n, k = 5, 160, 96
    A = rng.standard_normal((batch, n, k))
    B = rng.standard_normal((batch, k, n))
    Cin = rng.standard_normal((batch, n, n))
    C1 = pkg.batched_gemm(A, B, Cin=Cin, alpha=-0.37, beta=1.5, diag=0.25)
    ref = -0.37 * _exact(A, B) + 1.5 * Cin.astype(np.longdouble) + 0.25 * np.eye(n)
    bound = 4 * U * (0.37 * (np.abs(A) @ np.abs(B)) + 1.5 * np.abs(Cin) + 0.25 * np.eye(n))
    assert np.all(np.abs(C1.astype(np.longdouble) - ref).astype(np.float64) <= bound)
    pkg.set_emulation_scratch(3 << 20)                    # about one batch entry per chunk
    C2 = pkg.batched_gemm(A, B, Cin=Cin, alpha=-0.37, beta=1.5, diag=0.25)
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
    C = pkg.batched_gemm(A, B, Cin=Cin, alpha=alpha, beta=beta or 0.0, diag=diag)
    ref = alpha * _exact(A, B) + diag * np.eye(m, n)
    bound = 4 * U * (abs(alpha) * (np.abs(A) @ np.abs(B)) + abs(diag) * np.eye(m, n))
    if Cin is not None:
        ref = ref + beta * Cin.astype(np.longdouble)
        bound = bound + 4 * U * beta * np.abs(Cin)
    err = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
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
    C = pkg.batched_gemm(A, B)
    ref = _exact(A, B)
    if scale < 1:
        bound = 4 * U * (np.abs(A) @ np.abs(B)) + 2.0 ** -1074
        err = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
        assert np.all(err <= bound), (err / bound).max()
        assert np.all(np.abs(C) < 2.2250738585072014e-308)
    else:
        big = np.abs(ref) > np.longdouble("1e309")
        assert big.mean() > 0.9
        with np.errstate(over="ignore"):
            sign = np.sign(ref[big].astype(np.float64))
        assert np.all(np.isinf(C[big])) and np.all(np.sign(C[big]) == sign)
        small = np.abs(ref) < np.longdouble("1e307")
        bound = 4 * U * (np.abs(A).astype(np.longdouble) @ np.abs(B).astype(np.longdouble))
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
    C = pkg.batched_gemm(A, G, Cin=Cin, beta=0.5, mode=1)
    ref = _exact(A, G) + 0.5 * Cin.astype(np.longdouble)
    low = np.tril(np.ones((n, n), dtype=bool), -1)
    bound = 4 * U * ((np.abs(A) @ np.abs(G)) + 0.5 * np.abs(Cin))
    err = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err[:, low] <= bound[:, low])
    assert np.array_equal(C, -np.swapaxes(C, 1, 2))
    assert np.all(np.diagonal(C, axis1=1, axis2=2) == 0.0)
    # without Cin (the plain product's store pass)
    C0 = pkg.batched_gemm(A, G, mode=1)
    err0 = np.abs(C0.astype(np.longdouble) - _exact(A, G)).astype(np.float64)
    assert np.all(err0[:, low] <= 4 * U * (np.abs(A) @ np.abs(G))[:, low])
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
    C = pkg.batched_gemm(A, G, alpha=alpha, mode=mode, b_antisym=True)
    ref = alpha * _exact(A, G)
    bound = 4 * U * abs(alpha) * (np.abs(A) @ np.abs(G))
    err = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
    sel = np.tril(np.ones((n, n), dtype=bool), -1) if mode == 1 else np.ones((n, n), dtype=bool)
    assert np.all(err[:, sel] <= bound[:, sel]), (err / np.maximum(bound, 1e-300))[:, sel].max()
    if mode == 1:
        assert np.array_equal(C, -np.swapaxes(C, 1, 2))


def test_gauss_jordan_mode_matches_native_semantics(pkg):
    """Columns of the panel stay as they were; rows of the panel start from 0."""
    rng = np.random.default_rng(11)
    batch, n, k0, b = 2, 192, 64, 32
    A = rng.standard_normal((batch, n, b))
    B = rng.standard_normal((batch, b, n))
    W = rng.standard_normal((batch, n, n))
    C = pkg.batched_gemm(A, B, Cin=W, beta=1.0, mode=2, gj=(k0, b), C=W)
    pkg.set_fp64_gemm_path(pkg.FP64_FMA)
    Cn = pkg.batched_gemm(A, B, Cin=W, beta=1.0, mode=2, gj=(k0, b), C=W)
    pkg.set_fp64_gemm_path(pkg.FP64_EMULATED)
    cols = np.arange(n)
    panel = (cols >= k0) & (cols < k0 + b)
    assert np.array_equal(C[:, :, panel], W[:, :, panel])
    ref = _exact(A, B) + W.astype(np.longdouble)
    ref[:, k0:k0 + b, :] -= W[:, k0:k0 + b, :]
    bound = 4 * U * ((np.abs(A) @ np.abs(B)) + np.abs(W))
    err = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err[:, :, ~panel] <= bound[:, :, ~panel])
    # the native product is within its own K-term bound of the same value
    base = (np.abs(A) @ np.abs(B)) + np.abs(W)
    assert np.all(np.abs(C - Cn)[:, :, ~panel] <= (4 + b) * U * base[:, :, ~panel])


@pytest.mark.parametrize("n,batch", [(12, 3), (84, 2), (200, 1), (512, 2)])
def test_inverse_emulated(pkg, n, batch):
    rng = np.random.default_rng(300 + n)
    X = rng.standard_normal((batch, n, n))
    S = X - np.swapaxes(X, 1, 2)
    inv, ld = pkg.batched_inverse(S)
    for b in range(batch):
        ref = np.linalg.inv(S[b])
        assert np.abs(inv[b] - ref).max() < 1e-9 * np.abs(ref).max()
        assert abs(ld[b] - np.linalg.slogdet(S[b])[1]) < 1e-10 * max(1.0, abs(ld[b]))


@pytest.mark.parametrize("n,batch", [(6, 3), (66, 2), (256, 1)])
def test_pfaffian_emulated(pkg, n, batch):
    rng = np.random.default_rng(400 + n)
    Y = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    Y = Y - np.swapaxes(Y, 1, 2)
    ph, la = pkg.batched_pfaffian(Y)
    for b in range(batch):
        rph, rla = orc.pfaffian_log(Y[b])
        assert abs(la[b] - rla) < 1e-10 * max(1.0, abs(rla))
        assert abs(ph[b] - rph) < 1e-10


STEP_CASES = [
    # (n_bath, U, eps, V, M, seed, parity, channels)
    (15, 2.0, -1.0, 0.5, 4, 1, 1, 1),          # n = 64
    (40, 4.0, -2.0, 0.5, 6, 13, 1, 1),         # n = 164: several tiles
    (3, 2.0, -1.0, 0.5, 3, 11, -1, 2),         # two channels, odd parity, n = 28
]


@pytest.mark.parametrize("case", STEP_CASES)
def test_step_matches_oracle(pkg, case):
    """One step on the emulated path against the oracle, at the FP64 path's bars."""
    nb, Uc, e, V, M, seed, par, nc = case
    p = inp.AndersonParams(n_bath=nb, U=Uc, eps_d=e, V=V, n_channels=nc)
    g, lam = inp.initial_state(p.n_modes, M, seed, par)
    s = pkg.Solver(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels), g, lam, dtau=0.05,
                   parity=par)
    E = s.step(1)[0, 0]
    Gg, hg = s.pair_matrices()
    dg = s.derivative()
    g1, _ = s.get_state()
    s.close()
    model = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels)
    Eo, lo, Go, ho = orc.energy(model, list(g))
    do = orc.eom(model, list(g), Go, ho, Eo, lo)
    assert abs(E - Eo) <= 1e-10 * abs(Eo)
    assert np.abs(Gg - Go).max() <= 1e-10 * np.abs(Go).max()
    assert np.abs(hg - ho).max() <= 1e-10 * np.abs(ho).max()
    for mu in range(M):
        rt = 1e-10 + 50.0 * U * np.abs(lo).max() / max(abs(lo[mu]), 1e-300)
        assert np.abs(dg[mu] - do[mu]).max() <= rt * np.abs(do[mu]).max(), mu
        go = orc.purify(orc.orthogonal_step(g[mu], do[mu], 0.05))
        assert np.abs(g1[mu] - go).max() <= 1e-9 + 0.05 * rt * np.abs(do[mu]).max(), mu
        assert np.abs(g1[mu] @ g1[mu] + np.eye(2 * p.n_modes)).max() < 1e-12


def test_trajectory_and_mixed_form(pkg):
    """20 steps of the small workload on the emulated path against the oracle,
    and the TF32 form with emulated FP64 products against the TF32 form with
    native ones (same tensor-core products: agreement to FP64 rounding growth)."""
    w = inp.SMALL
    p = w.model
    g, lam = inp.initial_state(p.n_modes, w.rank, w.seed, w.parity)
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    s = pkg.Solver(m, g, lam, dtau=w.dtau)
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
        pkg.set_fp64_gemm_path(path)
        s = pkg.Solver(mq, gq, None, precision=1)
        out.append(s.step(3)[0])
        s.close()
    assert np.abs(out[0] - out[1]).max() <= 1e-9 * np.abs(out[1]).max()


@pytest.mark.parametrize("cmode", [0, 1])
def test_step_with_negligible_amplitudes(pkg, cmode):
    """Seeded random states at n = 164, M = 6: one state carries the weight and
    the other amplitudes are 1e-12 .. 3e-11 of it.  The decoupling constant of
    Sec. III A divides by the amplitude, so dGamma of such a state is fixed only
    to about kappa u max|lambda| / |lambda_mu| relative, with kappa the
    conditioning of the amplitude problem (G, h).  G, h and E still match the
    oracle at 1e-10; dGamma is held to 200 u max|lambda| / |lambda_mu|: with
    the phase form of c_mu, FP64 products on the FMA pipe reach 27 of that factor
    on this case and emulated ones 82, the difference being only where their
    roundings fall."""
    p = inp.AndersonParams(n_bath=40, U=4.0, eps_d=-2.0, V=0.5)
    g, lam = inp.initial_state(p.n_modes, 6, 13, 1)
    s = pkg.Solver(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, lam, cmode=cmode)
    E = s.step(1)[0, 0]
    Gg, hg = s.pair_matrices()
    dg = s.derivative()
    s.close()
    model = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V)
    Eo, lo, Go, ho = orc.energy(model, list(g))
    do = orc.eom(model, list(g), Go, ho, Eo, lo, cmode)
    assert abs(E - Eo) <= 1e-10 * abs(Eo)
    assert np.abs(Gg - Go).max() <= 1e-10 * np.abs(Go).max()
    assert np.abs(hg - ho).max() <= 1e-10 * np.abs(ho).max()
    assert np.abs(lo).min() < 1e-10 * np.abs(lo).max()           # the case is what it claims
    for mu in range(6):
        rt = 1e-10 + 200.0 * U * np.abs(lo).max() / abs(lo[mu])
        assert np.abs(dg[mu] - do[mu]).max() <= rt * np.abs(do[mu]).max(), mu
