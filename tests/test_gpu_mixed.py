"""Mixed-precision forms (tensor-core products of the equation of motion)
against the FP64 oracle (GPU).  The factorisations, the phase Pfaffian, the
Wick energies and the re-purification stay FP64, so the energy of a given
set of states is FP64-exact; only dGamma/ds (hence the trajectory) carries
the products' rounding.  Stated tolerances, with the values measured on a
GB300 in brackets: dGamma relative to its largest entry: TF32 1e-2 (2.9e-4),
BF16 6e-2 (2.3e-3), 3xTF32 1e-5 (1.9e-6); energy after 20 steps of the small
workload, relative: TF32 2e-4 (2.9e-5), BF16 2e-3 (5.7e-5), 3xTF32 1e-7
(4.5e-8)."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu

DG_TOL = {1: 1e-2, 2: 6e-2, 3: 1e-5}
E_TOL = {1: 2e-4, 2: 2e-3, 3: 1e-7}
# the state update of the TF32 and BF16 forms (exponential on the tensor cores, FP64 sums
# and purification; 3xTF32 updates in FP64): deviation from the exact step, relative to the
# step ds max|dGamma|.  Measured: TF32 3.8e-4, BF16 2.8e-3.
UPD_TOL = {1: 3e-3, 2: 2e-2, 3: 1e-9}


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def _solver(pkg, p, g, lam, prec, dtau=0.05, parity=1):
    m = pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels)
    return pkg.Solver(m, g, lam, dtau=dtau, precision=prec, parity=parity)


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mixed_derivative_and_energy(pkg, prec):
    p = inp.AndersonParams(n_bath=40, U=4.0, eps_d=-2.0, V=0.5)
    rng = np.random.default_rng(31)
    g = inp.clustered_pure_gammas(p.n_modes, 6, rng, 1, spread=1.0)
    lam = inp.random_amplitudes(6, rng)
    s = _solver(pkg, p, g, lam, prec)
    E = s.step(1)[0, 0]
    dg = s.derivative()
    model = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V)
    Eo, lo, Go, ho = orc.energy(model, list(g))
    do = orc.eom(model, list(g), Go, ho, Eo, lo)
    assert abs(E - Eo) <= 1e-10 * abs(Eo)          # energy of the given states: FP64 parts only
    errs = [np.abs(a - b).max() / np.abs(b).max() for a, b in zip(dg, do)]
    print(f"precision {prec}: dGamma relative error max {max(errs):.3e}")
    assert max(errs) < DG_TOL[prec]


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mixed_trajectory_energy(pkg, prec):
    w = inp.SMALL
    p = w.model
    g, lam = inp.initial_state(p.n_modes, w.rank, w.seed, w.parity)
    s = _solver(pkg, p, g, lam, prec, dtau=w.dtau)
    E = s.step(20)[0]
    s64 = _solver(pkg, p, g, lam, 0, dtau=w.dtau)
    E64 = s64.step(20)[0]
    rel = np.abs(E - E64).max() / np.abs(E64).max()
    print(f"precision {prec}: energy relative deviation over 20 steps {rel:.3e} (E20 = {E[-1]:.10f} vs {E64[-1]:.10f})")
    assert rel < E_TOL[prec]
    gg, _ = s.get_state()
    n = 2 * p.n_modes
    for G in gg:
        assert np.abs(G @ G + np.eye(n)).max() < 1e-12     # purity kept in FP64


@pytest.mark.parametrize("prec", [1, 2, 3])
def test_mixed_update_against_exact_step(pkg, prec):
    """Gamma after one step equals the exact orthogonal step (oracle expm) taken with
    the GPU's own dGamma, to the tensor-core rounding of the step's size; the
    result is pure to FP64 rounding."""
    p = inp.AndersonParams(n_bath=40, U=4.0, eps_d=-2.0, V=0.5)       # n = 164: ragged tiles
    rng = np.random.default_rng(33)
    g = inp.clustered_pure_gammas(p.n_modes, 5, rng, 1, spread=1.0)
    lam = inp.random_amplitudes(5, rng)
    s = _solver(pkg, p, g, lam, prec, dtau=0.2)
    s.step(1)
    dg = s.derivative()
    g1, _ = s.get_state()
    n = 2 * p.n_modes
    errs = []
    for mu in range(5):
        go = orc.purify(orc.orthogonal_step(g[mu], dg[mu], 0.2))
        errs.append(np.abs(g1[mu] - go).max() / (0.2 * np.abs(dg[mu]).max()))
        assert np.abs(g1[mu] @ g1[mu] + np.eye(n)).max() < 1e-12
    print(f"precision {prec}: update deviation relative to the step {max(errs):.3e}")
    assert max(errs) < UPD_TOL[prec]
