"""The paper's printed ground-state energy of the L = 500 single-impurity Anderson
model (tests/golden/siam_L500_E_star.txt, Sec. IV A, Fig. 1) against rigorous
bounds the oracle computes for the model this repository builds at the same
parameters.  With eps_d = -U/2,
    H = H_0(eps_d = 0) - U/4 + U (n_up - 1/2)(n_dn - 1/2),
and U (n_up - 1/2)(n_dn - 1/2) >= -U/4, so the exact ground energy E_0 is at least
the ground energy of the free model H_0(0) less U/2; it is at most <H> in any
state, here the free model's ground state (a single Gaussian, +-A|A|^-1).  The
estimate E* must lie in that window of width U/4 (it estimates E_0 to 4e-7): a
wrong hybridisation, level, sign or constant in the model map moves the window
off it."""
import os

import numpy as np

from oracle import sgs_oracle as orc

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "siam_L500_E_star.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _polar(A):
    Uu, _, Vh = np.linalg.svd(A)
    P = Uu @ Vh
    return 0.5 * (P - P.T)


def test_paper_energy_within_rigorous_bounds():
    g = _golden()
    L, U, t = int(g["L"]), g["U"], g["t"]
    V = np.sqrt(U / g["U_over_Gamma"] * t)                # Gamma = t'^2 / t = U / 5
    model = orc.anderson_model(L - 1, U, -U / 2, V, t)     # L sites: the impurity and L - 1 bath sites
    free = orc.anderson_model(L - 1, 0.0, 0.0, V, t)
    P = _polar(free.A)
    e_free = min(orc.wick_energy_density(free, s * P).real for s in (1.0, -1.0))
    lower = e_free - U / 2
    upper = min(orc.wick_energy_density(model, s * P).real for s in (1.0, -1.0))
    assert abs(upper - lower - U / 4) < 1e-9               # <n_up n_dn> = 1/4 in the symmetric free state
    assert lower - 4 * g["sigma"] <= g["E_star"] <= upper + 4 * g["sigma"]
