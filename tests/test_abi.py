"""The C-ABI library builds, loads and exports every function include/sgs.h
declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sgs.h")
LIB = os.path.join(ROOT, "paper_2105_01088_gb300", "libsgs.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(sgs_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2105_01088_gb300 import build as b
        b.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_four_calls():
    names = declared_functions()
    for n in ("sgs_init", "sgs_step", "sgs_energy", "sgs_correlator"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_signatures_cover_header():
    import paper_2105_01088_gb300 as pkg
    assert set(declared_functions()) == set(pkg.SIGNATURES)


def test_builder_matches_oracle_builder():
    import numpy as np
    import paper_2105_01088_gb300 as pkg
    from oracle import sgs_oracle as orc
    for args in ((15, 2.0, -1.0, 0.5, 1.0, 0.0, 1), (4, 8.0, -4.0, 0.6, 1.0, 0.1, 2)):
        nb, U, e, V, t, mu, nc = args
        m = pkg.build_anderson(nb, U, e, V, t, mu, nc)
        o = orc.anderson_model(nb, U, e, V, t, mu, nc)
        assert np.array_equal(m.A, o.A)
        assert abs(m.e_const - o.e_const) < 1e-12
        mono = orc.antisymmetrise_monomials([(tuple(m.quartic_idx[0]), m.quartic_val[0])])
        assert sorted(mono) == sorted(o.quartic)


def test_kondo_builder_matches_oracle_builder():
    """The library writes H_J from the closed form of the spin operators; the
    oracle expands S_imp . S_alpha(1) with its fermion-operator algebra."""
    import numpy as np
    import paper_2105_01088_gb300 as pkg
    from oracle import sgs_oracle as orc
    for L, J, t in ((2, 1.3, 0.5), (5, 0.7, 0.5), (4, 2.0, 1.0)):
        m = pkg.build_2ck(L, J, t)
        o = orc.two_channel_kondo_model(L, J, t)
        assert m.n == o.n == 8 * L
        assert np.array_equal(m.A, o.A) and m.e_const == o.e_const == 0.0
        mono = orc.antisymmetrise_monomials([(tuple(i), v) for i, v in zip(m.quartic_idx, m.quartic_val)])
        got = dict(mono)
        ref = dict(o.quartic)
        assert set(got) == set(ref) and max(abs(got[k] - ref[k]) for k in ref) < 1e-15


def test_invalid_arguments_are_rejected_without_gpu_work():
    import numpy as np
    import paper_2105_01088_gb300 as pkg
    m = pkg.build_anderson(3, 2.0, -1.0, 0.5)
    g = np.zeros((2, m.n, m.n))
    with pytest.raises(pkg.SGSError) as e:
        pkg.Solver(m, g, parity=3)
    assert e.value.status == 1
    with pytest.raises(pkg.SGSError):
        pkg.Solver(m, np.zeros((65, m.n, m.n)))
