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


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mixed_step_is_deterministic(pkg, prec):
    """The tensor-core products have a fixed reduction order: two runs of the same
    mixed-precision steps (ragged 128-tiles at n = 164) agree bit for bit."""
    import sgs_inputs as inp
    p = inp.AndersonParams(n_bath=40, U=4.0, eps_d=-2.0, V=0.5)
    rng = np.random.default_rng(3)
    g = inp.clustered_pure_gammas(p.n_modes, 5, rng, 1, spread=1.0)
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    out = []
    for _ in range(2):
        s = pkg.Solver(m, g, None, precision=prec)
        E = s.step(2)
        out.append((E, s.derivative(), s.get_state()[0]))
        s.close()
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)
