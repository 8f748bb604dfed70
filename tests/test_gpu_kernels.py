"""Building blocks of the CUDA path against plain FP64 references (GPU), on
both arithmetics of the FP64 products (0 emulated on the tensor cores, 1 FP64
FMA)."""
import numpy as np
import pytest

from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


PATHS = [0, 1]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n,batch", [(8, 3), (64, 2), (100, 2), (130, 1), (512, 2)])
def test_gemm_matches_numpy(pkg, n, batch, path):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((batch, n, n))
    B = rng.standard_normal((batch, n, n))
    C = pkg.batched_gemm(A, B, fp64_path=path)
    ref = A @ B
    assert np.abs(C - ref).max() < 1e-12 * np.abs(ref).max() * np.sqrt(n)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n,batch", [(4, 2), (12, 3), (64, 2), (84, 2), (200, 1), (512, 2)])
def test_inverse_matches_numpy(pkg, n, batch, path):
    rng = np.random.default_rng(100 + n)
    X = rng.standard_normal((batch, n, n))
    S = X - np.swapaxes(X, 1, 2)            # the method inverts skew matrices
    inv, ld = pkg.batched_inverse(S, fp64_path=path)
    for b in range(batch):
        ref = np.linalg.inv(S[b])
        assert np.abs(inv[b] - ref).max() < 1e-9 * np.abs(ref).max()
        assert abs(ld[b] - np.linalg.slogdet(S[b])[1]) < 1e-10 * max(1.0, abs(ld[b]))
    # general (non-skew) matrices too
    G = rng.standard_normal((1, n, n)) + n ** 0.5 * np.eye(n)
    inv, _ = pkg.batched_inverse(G, fp64_path=path)
    assert np.abs(inv[0] @ G[0] - np.eye(n)).max() < 1e-10


@pytest.mark.parametrize("path", PATHS)
def test_inverse_flags_singular(pkg, path):
    S = np.zeros((1, 6, 6))
    with pytest.raises(pkg.SGSError) as e:
        pkg.batched_inverse(S, fp64_path=path)
    assert e.value.status == 3


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n,batch", [(2, 2), (6, 3), (32, 2), (66, 2), (130, 1), (256, 1)])
def test_pfaffian_matches_oracle(pkg, n, batch, path):
    rng = np.random.default_rng(200 + n)
    Y = rng.standard_normal((batch, n, n)) + 1j * rng.standard_normal((batch, n, n))
    Y = Y - np.swapaxes(Y, 1, 2)
    ph, la = pkg.batched_pfaffian(Y, fp64_path=path)
    for b in range(batch):
        rph, rla = orc.pfaffian_log(Y[b])
        assert abs(la[b] - rla) < 1e-10 * max(1.0, abs(rla))
        assert abs(ph[b] - rph) < 1e-10


def test_shared_memory_limits_raised_on_the_current_device(pkg):
    """Kernels with large tiles get their dynamic shared-memory limit raised on every
    device they run on: the limit in force equals the opt-in maximum less the kernel's
    static shared memory."""
    for lim, exp in pkg.smem_limits():
        assert lim == exp and lim > 200 * 1024
