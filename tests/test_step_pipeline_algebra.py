"""One imaginary-time step (Sec. III C) composed from the CPU transcriptions of
the CUDA path's kernels, against the oracle's step:

  pair pass (`test_pair_pass_algebra.composed_gh`) -> amplitude solve
  (`test_amplitude_algebra.amp_solve`) -> equation of motion
  (`test_eom_pipeline_algebra.composed_eom`) -> FP64 update with one
  Newton-Schulz iteration (`test_update_algebra.fp64_update`),

for both parities and both forms of c_mu, over two consecutive steps."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc
from test_amplitude_algebra import amp_solve
from test_eom_pipeline_algebra import composed_eom
from test_pair_pass_algebra import composed_gh
from test_update_algebra import fp64_update


def composed_step(model, gammas, ds, parity, cmode):
    G, h = composed_gh(model, gammas, parity)
    E, lam = amp_solve(G, h)
    dGs = composed_eom(model, gammas, cmode, amplitudes=(G, h, E, lam))
    return E, [fp64_update(g, d, ds)[0] for g, d in zip(gammas, dGs)]


@pytest.mark.parametrize("parity,cmode", [(1, orc.C_INVERSE), (-1, orc.C_PHASE)])
def test_composed_step_equals_the_oracle_step(parity, cmode):
    model = orc.anderson_model(3, 2.0, -1.0, 0.5)
    gammas, _ = inp.initial_state(model.N, 4, 7, parity)
    g_ours, g_ref = list(gammas), list(gammas)
    for _ in range(2):
        E, g_ours = composed_step(model, g_ours, 0.05, parity, cmode)
        Eo, _, g_ref = orc.sgs_step(model, g_ref, 0.05, cmode)
        assert abs(E - Eo) < 1e-11 * abs(Eo)
        assert max(np.abs(a - b).max() for a, b in zip(g_ours, g_ref)) < 1e-10
