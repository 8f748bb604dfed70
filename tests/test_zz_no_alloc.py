"""The allocation-free batched inverse (for callers that must not allocate
device memory during a call) agrees with the allocating batched inverse, on
two calls in a row that share its static scratch array.  The test itself
owns the device buffers it passes in."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RTOL = 1e-10


def test_static_inverse_matches_allocating_inverse_twice():
    torch = pytest.importorskip("torch")
    import paper_2105_01088_gb300 as pkg

    rng = np.random.default_rng(2024)
    for n, batch in ((200, 3), (512, 4), (84, 2)):
        for call in range(2):   # second call reuses the scratch left by the first
            X = rng.standard_normal((batch, n, n))
            S = X - np.swapaxes(X, 1, 2)
            ref_inv, ref_ld = pkg.batched_inverse(S)
            dS = torch.from_numpy(S).cuda()
            dinv = torch.full_like(dS, float("nan"))
            dld = torch.full((batch,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            pkg.batched_inverse_static(dS.data_ptr(), dinv.data_ptr(), dld.data_ptr(), n, batch)
            inv = dinv.cpu().numpy()
            ld = dld.cpu().numpy()
            for b in range(batch):
                scale = np.abs(ref_inv[b]).max()
                assert np.abs(inv[b] - ref_inv[b]).max() <= RTOL * scale, (n, call, b)
                assert abs(ld[b] - ref_ld[b]) <= RTOL * max(1.0, abs(ref_ld[b])), (n, call, b)


def test_static_inverse_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    import paper_2105_01088_gb300 as pkg

    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    for n, batch in ((1025, 1), (512, 65), (0, 1)):
        with pytest.raises(pkg.SGSError) as e:
            pkg.batched_inverse_static(d.data_ptr(), d.data_ptr(), d.data_ptr(), n, batch)
        assert e.value.status == 1
