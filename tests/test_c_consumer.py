"""The C ABI from C (CPU): include/sgs.h compiles as strict C99 and as C++17 on
its own, and a C99 program (tests/c_consumer.c) linked against libsgs.so calls
the host-side model builders.  What it prints matches the oracle's models, and
the library rejects bad arguments with -1."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import sgs_oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2105_01088_gb300")
LIB = os.path.join(PKG, "libsgs.so")
INC = os.path.join(ROOT, "include")

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None or shutil.which("g++") is None,
                                reason="needs gcc and g++")


@pytest.fixture(scope="module")
def consumer(tmp_path_factory):
    if not os.path.exists(LIB):
        from paper_2105_01088_gb300 import build as b
        b.build()
    exe = str(tmp_path_factory.mktemp("c") / "c_consumer")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", INC,
           os.path.join(ROOT, "tests", "c_consumer.c"), "-L", PKG, "-lsgs", f"-Wl,-rpath,{PKG}", "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


@pytest.mark.parametrize("compiler,std,lang", [("gcc", "-std=c99", "c"), ("g++", "-std=c++17", "c++")])
def test_header_compiles_alone(compiler, std, lang, tmp_path):
    r = subprocess.run([compiler, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", lang,
                        os.path.join(INC, "sgs.h")], capture_output=True, text=True, cwd=tmp_path)
    assert r.returncode == 0, r.stderr


def _run(exe, *args):
    r = subprocess.run([exe, *[str(a) for a in args]], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    N, e_const, A_entries, quartic = None, None, [], []
    for line in r.stdout.splitlines():
        f = line.split()
        if f[0] == "N":
            N = int(f[1])
        elif f[0] == "e_const":
            e_const = float(f[1])
        elif f[0] == "A":
            A_entries.append((int(f[1]), int(f[2]), float(f[3])))
        elif f[0] == "Q":
            quartic.append((tuple(int(x) for x in f[1:5]), float(f[5])))
    n = 2 * N
    A = np.zeros((n, n))
    for k, l, v in A_entries:
        A[k, l] = v
    return N, A, e_const, quartic


@pytest.mark.parametrize("args", [(15, 1, 2.0, -1.0, 0.5, 1.0, 0.0), (4, 2, 8.0, -4.0, 0.6, 1.0, 0.1)])
def test_anderson_from_c_matches_the_oracle(consumer, args):
    nb, nc, U, e, V, t, mu = args
    N, A, e_const, quartic = _run(consumer, "anderson", *args)
    o = orc.anderson_model(nb, U, e, V, t, mu, nc)
    assert N == o.N
    assert np.array_equal(A, o.A)
    assert abs(e_const - o.e_const) < 1e-12
    assert sorted(orc.antisymmetrise_monomials(quartic)) == sorted(o.quartic)


@pytest.mark.parametrize("L,J,t", [(2, 1.3, 0.5), (5, 0.7, 0.5)])
def test_two_channel_kondo_from_c_matches_the_oracle(consumer, L, J, t):
    N, A, e_const, quartic = _run(consumer, "2ck", L, J, t)
    o = orc.two_channel_kondo_model(L, J, t)
    assert N == o.N and np.array_equal(A, o.A) and e_const == o.e_const == 0.0
    got = dict(orc.antisymmetrise_monomials(quartic))
    ref = dict(o.quartic)
    assert set(got) == set(ref) and max(abs(got[k] - ref[k]) for k in ref) < 1e-15


def test_bad_arguments_from_c(consumer):
    r = subprocess.run([consumer, "bad"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["anderson", "-1", "2ck", "-1"]
