"""Continuous batching on the GPU: a slot's results are the same alone and
in a mix whose other slots are admitted and retired around it; admission
follows the HBM budget; the request loop reproduces solo solves."""
import numpy as np
import pytest

import sgs_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2105_01088_gb300 as p
    return p


def _req(pkg, n_bath, M, seed, U=2.0, V=0.5):
    p = inp.AndersonParams(n_bath=n_bath, U=U, eps_d=-U / 2, V=V)
    g, lam = inp.initial_state(p.n_modes, M, seed, 1 if (n_bath + 1) % 2 == 0 else -1)
    return pkg.build_anderson(n_bath, U, -U / 2, V), g, lam, 1 if (n_bath + 1) % 2 == 0 else -1


@pytest.mark.parametrize("precision", [0, 1])
def test_alone_equals_mix(pkg, precision):
    import torch
    stream = torch.cuda.Stream()
    A = _req(pkg, 15, 4, 1)
    B = _req(pkg, 23, 6, 2, U=3.0)
    C = _req(pkg, 11, 3, 3, U=1.0)
    alone = pkg.Solver(stream=stream)
    a = alone.admit(A[0], A[1], A[2], 0.05, precision, 0, A[3])
    Ea = alone.step(25)[a]
    ga, _ = alone.get_state(a)
    alone.close()
    mix = pkg.Solver(stream=stream)
    b = mix.admit(B[0], B[1], B[2], 0.05, precision, 0, B[3])
    mix.step(3)
    a2 = mix.admit(A[0], A[1], A[2], 0.05, precision, 0, A[3])
    E1 = mix.step(10)[a2]
    c = mix.admit(C[0], C[1], C[2], 0.05, precision, 0, C[3])
    E2 = mix.step(5)[a2]
    mix.retire(b)
    E3 = mix.step(10)[a2]
    gm, _ = mix.get_state(a2)
    mix.close()
    assert np.array_equal(np.concatenate([E1, E2, E3]), Ea)
    assert np.array_equal(gm, ga)


def test_admission_by_budget(pkg):
    A = _req(pkg, 15, 4, 1)
    probe = pkg.Solver()
    probe.admit(A[0], A[1], A[2], parity=A[3])
    one = probe.bytes_in_use()
    probe.close()
    s = pkg.Solver(hbm_budget=int(1.5 * one))
    x = s.admit(A[0], A[1], A[2], parity=A[3])
    with pytest.raises(pkg.SGSError) as e:
        s.admit(A[0], A[1], A[2], parity=A[3])
    assert e.value.status == 2
    s.retire(x)
    assert s.bytes_in_use() < one
    y = s.admit(A[0], A[1], A[2], parity=A[3])
    assert y == 1 and s.step(1).shape == (2, 1)
    s.close()


def test_request_loop_matches_solo_solves(pkg):
    import torch
    from paper_2105_01088_gb300.serving import Request, ServingLoop, latency_stats
    stream = torch.cuda.Stream()
    reqs = []
    for i, (t, p, M, seed, par) in enumerate(inp.serving_requests(200.0, 6, seed=9, n_bath=(7, 15), ranks=(3, 4))):
        g, lam = inp.initial_state(p.n_modes, M, seed, par)
        reqs.append(Request(i, t, pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, lam, par))
    solver = pkg.Solver(stream=stream)
    loop = ServingLoop(solver, tol=1e-8, max_steps=60, keep_energies=True)
    res = loop.run(reqs)
    solver.close()
    assert len(res) == 6
    st = latency_stats(res)
    assert st["p99_s"] >= st["p50_s"] > 0
    for r in res:
        solo = pkg.Solver(stream=stream)
        k = solo.admit(reqs[r.rid].model, reqs[r.rid].gamma0, reqs[r.rid].lambda0, parity=reqs[r.rid].parity)
        E = solo.step(r.steps)[k]
        solo.close()
        assert np.array_equal(E, np.array(r.energies))
