"""The seeded input generators (CPU): the counter-based generator against the
published known-answer vectors of Philox4x32-10, the seeded states' purity and
parity, and the library's own generation of the same states (host code, no GPU)."""
import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc


def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 (Salmon et al., SC11)."""
    cases = [((0, 0, 0, 0), 0, (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
             ((0xffffffff,) * 4, 0xffffffffffffffff, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
             ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0x299f31d0 << 32) | 0xa4093822,
              (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1))]
    for ctr, key, want in cases:
        got = inp.philox4x32(np.array([ctr], dtype=np.uint64), key)[0]
        assert tuple(int(v) for v in got) == want


@pytest.mark.parametrize("parity", [1, -1])
def test_seeded_states_are_pure_with_the_parity(parity):
    g, lam = inp.seeded_states(5, 3, 99, parity)
    for G in g:
        assert np.abs(G @ G + np.eye(10)).max() < 1e-13
        assert abs(orc.pfaffian(G) - parity) < 1e-12
    assert np.allclose(np.abs(lam), 1.0)
    g2, _ = inp.seeded_states(5, 3, 100, parity)
    assert np.abs(g - g2).max() > 0.1                     # another seed, other states


def test_library_generates_the_same_states():
    import paper_2105_01088_gb300 as pkg
    for N, M, seed, par in ((6, 3, 12345, 1), (16, 2, 2 ** 40 + 7, -1)):
        g1, l1 = pkg.seeded_states(N, M, seed, par)
        g2, l2 = inp.seeded_states(N, M, seed, par)
        assert np.abs(g1 - g2).max() < 1e-13 and np.abs(l1 - l2).max() < 1e-15
