"""tcgen05 tensor-core GEMM against numpy (GPU).  Bounds per operand type:
TF32 keeps 10 mantissa bits of each operand, BF16 7; each product then
errs by at most ~2 u_op relative, plus fp32 accumulation, so
|C - AB| <= c_kind * (|A| |B|) elementwise."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOUND = {0: 3e-3, 1: 1.6e-2, 2: 2e-5}


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("m,n,k,batch", [(128, 128, 32, 1), (256, 256, 512, 2), (300, 200, 104, 2), (64, 72, 8, 1)])
def test_tc_gemm_matches_numpy(pkg, kind, m, n, k, batch):
    rng = np.random.default_rng(m + n + k + kind)
    A = rng.standard_normal((batch, m, k))
    B = rng.standard_normal((batch, k, n))
    C = pkg.batched_gemm_tc(A, B, kind)
    ref = A @ B
    bound = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(C - ref) <= BOUND[kind] * bound + 1e-30), np.abs(C - ref).max() / bound.max()
    # and the error is not trivially zero-tolerance satisfied: the result is a real product
    assert np.abs(ref).max() > 0 and np.abs(C - ref).max() < 0.05 * np.abs(ref).max()


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_tma_and_cp_async_staging_agree(pkg, kind):
    """The TMA-fed kernel (128-byte swizzle, mbarrier pipeline) and the
    cp.async-fed one issue the same MMA sequence: identical results, ragged
    tiles and K tails included."""
    rng = np.random.default_rng(kind + 5)
    A = rng.standard_normal((3, 300, 104))
    B = rng.standard_normal((3, 104, 200))
    pkg.set_tc_loader(True)
    C1 = pkg.batched_gemm_tc(A, B, kind)
    pkg.set_tc_loader(False)
    try:
        C2 = pkg.batched_gemm_tc(A, B, kind)
    finally:
        pkg.set_tc_loader(True)
    assert np.array_equal(C1, C2)
    assert np.all(np.abs(C1 - A @ B) <= BOUND[kind] * (np.abs(A) @ np.abs(B)) + 1e-30)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_persistent_tma_kernel_agrees(pkg, kind):
    """The persistent form (one CTA per SM looping over tiles, two TMEM
    accumulators) gives the one-tile-per-CTA results bit for bit: 240 ragged
    tiles over 152 SMs, so CTAs take one or two tiles and both accumulators."""
    rng = np.random.default_rng(kind + 11)
    A = rng.standard_normal((40, 300, 136))
    B = rng.standard_normal((40, 136, 200))
    pkg.set_tc_loader(True)
    C1 = pkg.batched_gemm_tc(A, B, kind)
    pkg.set_tc_loader(True, persistent=True)
    try:
        C2 = pkg.batched_gemm_tc(A, B, kind)
    finally:
        pkg.set_tc_loader(True)
    assert np.array_equal(C1, C2)
    assert np.all(np.abs(C1 - A @ B) <= BOUND[kind] * (np.abs(A) @ np.abs(B)) + 1e-30)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mixed_step_identical_under_both_stagings(pkg, prec):
    """The loader switch applies to the equation of motion's products (and the
    persistent form to the state update's TMA-fed products too).  All three
    stagings give identical steps."""
    import sgs_inputs as inp
    p = inp.AndersonParams(n_bath=40, U=4.0, eps_d=-2.0, V=0.5)        # n = 164: ragged 128-tiles
    rng = np.random.default_rng(3)
    g = inp.clustered_pure_gammas(p.n_modes, 5, rng, 1, spread=1.0)
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    out = []
    for tma, pers in ((True, False), (False, False), (True, True)):
        pkg.set_tc_loader(tma, persistent=pers)
        s = pkg.Solver(m, g, None, precision=prec)
        E = s.step(2)
        out.append((E, s.derivative(), s.get_state()[0]))
        s.close()
    pkg.set_tc_loader(True)
    for other in out[1:]:
        for x, y in zip(out[0], other):
            assert np.array_equal(x, y)
