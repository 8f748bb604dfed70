"""Health reporting and input validation (GPU): the purity residual, non-finite
count and Gram conditioning of the current states; admission rejects initial
states that are not finite or not antisymmetric."""
import numpy as np
import pytest

import sgs_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def test_health_after_steps(pkg):
    p = inp.AndersonParams(n_bath=20, U=3.0, eps_d=-1.5, V=0.7)
    rng = np.random.default_rng(5)
    g = inp.clustered_pure_gammas(p.n_modes, 4, rng, 1, spread=1.0)
    s = pkg.Solver(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, None)
    E = s.step(3)[0]
    h = s.health()
    Gm, _ = s.pair_matrices()
    s.close()
    assert h["purity_residual"] < 1e-12 and h["nonfinite"] == 0
    w = np.linalg.eigvalsh(Gm)
    assert abs(h["gram_eig_ratio"] - w.min() / w.max()) < 1e-10
    assert h["energy"] == E[-1]


def test_admission_rejects_bad_states(pkg):
    p = inp.AndersonParams(n_bath=7, U=2.0, eps_d=-1.0, V=0.5)
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    g, lam = inp.initial_state(p.n_modes, 2, 3, 1)
    s = pkg.Solver()
    for bad in (np.nan, np.inf):
        x = g.copy()
        x[1, 0, 3] = bad
        with pytest.raises(pkg.SGSError) as e:
            s.admit(m, x, lam)
        assert e.value.status == 1
    x = g.copy()
    x[0, 2, 5] += 1e-3                                  # no longer antisymmetric
    with pytest.raises(pkg.SGSError) as e:
        s.admit(m, x, lam)
    assert e.value.status == 1
    assert s.admit(m, g, lam) == 0                      # the context stays usable
    s.close()


@pytest.mark.parametrize("limit_ms", [1, 20])
def test_bounded_wait_runs_out_and_the_context_stays_usable(pkg, limit_ms):
    """A device wait on a flag that nothing sets gives up after its limit, records the
    timeout and returns: the call reports SGS_ETIMEOUT (5), the launch lasted about the
    limit, and the next library call on the device works."""
    import paper_2105_01088_gb300 as pkg
    st, ms = pkg.probe_wait(limit_ms * 1_000_000)
    assert st == 5
    assert 0.9 * limit_ms <= ms <= limit_ms + 50.0
    A = np.random.default_rng(1).standard_normal((1, 64, 64))
    C = pkg.batched_gemm(A, A)
    assert np.abs(C - A @ A).max() < 1e-12 * np.abs(A @ A).max() * 8
    assert pkg.probe_wait(10)[0] == 1               # limit below 1 us: rejected before any launch
