"""The allocation-free batched inverse, sgs_kernel_inverse_static, for callers
that must not allocate device memory during a call: a host program whose
device memory belongs entirely to another framework's pool, or a
latency-critical loop that cannot take cudaMalloc's implicit device
synchronisation.  Checked on two calls in a row that share its static scratch
array, against the allocating entry point (sgs_kernel_inverse on the same FP64
FMA products) and against numpy's inverse and log-determinant, up to the
documented limit n = 1024 (batch * n <= 32768); on the legacy default stream
and on a stream of its own; and for what it is for: after one warm-up call,
repeated calls change neither the device's free memory nor call the library's
allocation hook.  The test owns the device buffers it passes in."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def _skew(rng, batch, n):
    X = rng.standard_normal((batch, n, n))
    return X - np.swapaxes(X, 1, 2)


def _static(pkg, torch, S, stream=None):
    batch, n, _ = S.shape
    dS = torch.from_numpy(S).cuda()
    dinv = torch.full_like(dS, float("nan"))
    dld = torch.full((batch,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    pkg.batched_inverse_static(dS.data_ptr(), dinv.data_ptr(), dld.data_ptr(), n, batch,
                               stream.cuda_stream if stream is not None else None)
    return dinv.cpu().numpy(), dld.cpu().numpy()


def _check(inv, ld, S, ref_inv, ref_ld, tag):
    for b in range(S.shape[0]):
        scale = np.abs(ref_inv[b]).max()
        assert np.abs(inv[b] - ref_inv[b]).max() <= RTOL * scale, (tag, b)
        assert abs(ld[b] - ref_ld[b]) <= RTOL * max(1.0, abs(ref_ld[b])), (tag, b)
        # independent reference: numpy's LU inverse and log|det|
        npi = np.linalg.inv(S[b])
        assert np.abs(inv[b] - npi).max() <= 1e-9 * np.abs(npi).max(), (tag, b)
        assert abs(ld[b] - np.linalg.slogdet(S[b])[1]) <= RTOL * max(1.0, abs(ld[b])), (tag, b)


def test_static_inverse_matches_allocating_inverse_twice():
    torch = pytest.importorskip("torch")
    import paper_2105_01088_gb300 as pkg

    rng = np.random.default_rng(2024)
    for n, batch in ((200, 3), (512, 4), (84, 2), (1024, 2)):
        for call in range(2):   # the second call reuses the scratch the first left behind
            S = _skew(rng, batch, n)
            ref_inv, ref_ld = pkg.batched_inverse(S, fp64_path=pkg.FP64_FMA)
            inv, ld = _static(pkg, torch, S)
            _check(inv, ld, S, ref_inv, ref_ld, (n, call))


def test_static_inverse_at_the_batch_limit_on_its_own_stream():
    """batch * n = 32768 (the largest the scratch holds) at n = 1024, on a
    non-default stream, twice."""
    torch = pytest.importorskip("torch")
    import paper_2105_01088_gb300 as pkg

    rng = np.random.default_rng(7)
    stream = torch.cuda.Stream()
    for call in range(2):
        S = _skew(rng, 32, 1024)
        ref_inv, ref_ld = pkg.batched_inverse(S, fp64_path=pkg.FP64_FMA)
        inv, ld = _static(pkg, torch, S, stream)
        idx = [0, 13, 31] if call == 0 else [5, 30]
        _check(inv[idx], ld[idx], S[idx], ref_inv[idx], ref_ld[idx], call)


def test_static_inverse_allocates_nothing():
    torch = pytest.importorskip("torch")
    import paper_2105_01088_gb300 as pkg

    rng = np.random.default_rng(3)
    n, batch = 256, 4
    S = _skew(rng, batch, n)
    dS = torch.from_numpy(S).cuda()
    dinv = torch.empty_like(dS)
    dld = torch.empty((batch,), dtype=torch.float64, device="cuda")
    calls = []
    alloc_fn = pkg._ALLOC_FN(lambda nbytes, stream, user: calls.append(nbytes) or None)
    free_fn = pkg._FREE_FN(lambda ptr, user: calls.append(-1))
    pkg._lib.sgs_set_allocator(alloc_fn, free_fn, None)
    try:
        pkg.batched_inverse_static(dS.data_ptr(), dinv.data_ptr(), dld.data_ptr(), n, batch)   # warm-up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(5):
            pkg.batched_inverse_static(dS.data_ptr(), dinv.data_ptr(), dld.data_ptr(), n, batch)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
    finally:
        hooks = pkg._torch_hooks
        if hooks is not None:
            pkg._lib.sgs_set_allocator(hooks[0], hooks[1], None)
        else:
            pkg._lib.sgs_set_allocator(ctypes.cast(None, pkg._ALLOC_FN), ctypes.cast(None, pkg._FREE_FN), None)
    assert calls == []
    assert free1 == free0
    npi = np.linalg.inv(S[1])
    assert np.abs(dinv.cpu().numpy()[1] - npi).max() <= 1e-9 * np.abs(npi).max()


def test_static_inverse_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    import paper_2105_01088_gb300 as pkg

    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    for n, batch in ((1025, 1), (512, 65), (1024, 33), (0, 1)):
        with pytest.raises(pkg.SGSError) as e:
            pkg.batched_inverse_static(d.data_ptr(), d.data_ptr(), d.data_ptr(), n, batch)
        assert e.value.status == 1
