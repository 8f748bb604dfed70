"""The factorisation autotuner (GPU): it picks panel widths from the allowed
candidates, caches them per (n, rank, precision), and changes results only by
rounding."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def test_autotune_choices_cache_and_results(pkg):
    import torch
    p = inp.AndersonParams(n_bath=37, U=3.0, eps_d=-1.5, V=0.6)      # n = 152
    rng = np.random.default_rng(61)
    g = inp.clustered_pure_gammas(p.n_modes, 5, rng, 1, spread=1.0)
    lam = inp.random_amplitudes(5, rng)
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    st = torch.cuda.Stream()
    tuned = pkg.Solver(stream=st, autotune=True)
    k1 = tuned.admit(m, g, lam)
    gj, pf, src = tuned.tuning(k1)
    assert gj in (8, 16, 24, 32, 48, 64) and pf in (8, 12, 16, 24, 32) and src == 0
    k2 = tuned.admit(m, g[::-1].copy(), lam[::-1].copy())
    assert tuned.tuning(k2) == (gj, pf, 1)
    E = tuned.step(3)
    plain = pkg.Solver(m, g, lam, stream=st)
    assert plain.tuning(0)[2] == -1
    Ep = plain.step(3)[0]
    assert np.abs(E[k1] - Ep).max() <= 1e-12 * np.abs(Ep).max()
    Eo, _, _ = orc.run(orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V), list(g), 0.05, 3)
    assert np.abs(E[k1] - Eo).max() <= 1e-10 * np.abs(Eo).max()
    # rank growth re-tunes the new shape
    tuned.add_state(inp.random_generator(2 * p.n_modes, 0.2, rng), slot=k1)
    assert tuned.tuning(k1)[2] in (0, 1)
    tuned.close()
    plain.close()


def test_fixed_panel_widths(pkg):
    """Widths fixed after admission (reproducible profiles): any candidate within the
    scratch, results equal to the tuned instance's up to rounding; others refused."""
    import torch
    p = inp.AndersonParams(n_bath=37, U=3.0, eps_d=-1.5, V=0.6)      # n = 152
    rng = np.random.default_rng(62)
    g = inp.clustered_pure_gammas(p.n_modes, 4, rng, 1, spread=1.0)
    lam = inp.random_amplitudes(4, rng)
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V)
    st = torch.cuda.Stream()
    s = pkg.Solver(m, g, lam, stream=st, autotune=True)
    E0 = s.step(2)[0]
    s.close()
    s = pkg.Solver(m, g, lam, stream=st, autotune=True)
    s.set_panel_widths(24, 12)
    assert s.tuning(0) == (24, 12, 2)
    E1 = s.step(2)[0]
    assert np.abs(E1 - E0).max() <= 1e-12 * np.abs(E0).max()
    with pytest.raises(pkg.SGSError):
        s.set_panel_widths(28, 12)                     # not a candidate
    assert s.tuning(0) == (24, 12, 2)
    s.close()
