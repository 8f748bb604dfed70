"""The pair-sharded step on the GPU (sgs_shard_pairs / eom / update through
paper_2105_01088_gb300.sharded): ranks as separate processes on one GPU, the
two sums over ranks made by gloo through host memory (no kernel waits on
another rank).  Summed shares must reproduce the unsharded library step
(energies to 1e-12 relative, states to 1e-10) and the oracle; each rank's
share of (G, h) holds exactly its pairs and its states' diagonal."""
import os
import socket

import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc

pytestmark = pytest.mark.gpu
N_STEPS = 3


def _case():
    p = inp.AndersonParams(n_bath=20, U=3.0, eps_d=-1.5, V=0.7)          # n = 84: ragged tiles
    rng = np.random.default_rng(17)
    g = inp.clustered_pure_gammas(p.n_modes, 7, rng, 1, spread=1.0)      # order-one amplitudes
    return p, g


def _worker(rank, world, port, out_dir, fp64_path):
    import torch
    import torch.distributed as dist

    import paper_2105_01088_gb300 as pkg
    from paper_2105_01088_gb300.sharded import LibraryShard, ShardedStep
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        p, g = _case()
        s = pkg.Solver(fp64_path=fp64_path)
        s.admit(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, None, 0.05, shard=(rank, world))
        backend = LibraryShard(s)
        gh0 = backend.pairs().cpu().numpy().copy()             # this rank's share before any sum
        E = ShardedStep(backend).step(N_STEPS)
        gam, lam = s.get_state()
        s.close()
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), E=E, g=gam, gh0=gh0)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


@pytest.mark.parametrize("fp64_path", [0, 1])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_step_equals_unsharded(tmp_path, world, fp64_path):
    import torch.multiprocessing as mp

    import paper_2105_01088_gb300 as pkg
    from paper_2105_01088_gb300.sharded import local_pairs, own_states
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), fp64_path), nprocs=world, join=True)
    p, g = _case()
    s = pkg.Solver(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, None, dtau=0.05, fp64_path=fp64_path)
    E1 = s.step(N_STEPS)[0]
    g1, _ = s.get_state()
    s.close()
    Eo, _, go = orc.run(orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V), list(g), 0.05, N_STEPS)
    assert np.all(np.abs(E1 - Eo) <= 1e-10 * np.abs(Eo))
    M = len(g)
    shares = []
    for r in range(world):
        res = np.load(tmp_path / f"rank{r}.npz")
        assert np.all(np.abs(res["E"] - E1) <= 1e-12 * np.abs(E1)), (r, res["E"] - E1)
        assert np.abs(res["g"] - g1).max() <= 1e-10, r
        assert np.abs(res["g"] - np.stack(go)).max() <= 1e-9, r
        gh = res["gh0"].view(np.complex128).reshape(2, M, M)
        mask = np.zeros((M, M), bool)
        for a, b in local_pairs(M, r, world):
            mask[a, b] = mask[b, a] = True
        for mu in own_states(M, r, world):
            mask[mu, mu] = True
        assert np.all(gh[:, ~mask] == 0.0) and np.all(np.abs(gh[0][mask]) > 0.0), r
        shares.append(gh)
    # the shares add up to the whole (G, h) of the oracle at the initial states
    _, _, Go, ho = orc.energy(orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V), list(g))
    tot = np.sum(shares, axis=0)
    assert np.abs(tot[0] - Go).max() <= 1e-10 * np.abs(Go).max()
    assert np.abs(tot[1] - ho).max() <= 1e-10 * np.abs(ho).max()


def test_sharded_instance_refuses_the_whole_step():
    import paper_2105_01088_gb300 as pkg
    p, g = _case()
    s = pkg.Solver()
    s.admit(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, None, 0.05, shard=(0, 2))
    with pytest.raises(pkg.SGSError) as e:
        s.step(1)
    assert e.value.status == 1
    with pytest.raises(pkg.SGSError):
        s.correlator(pkg.SGS_CORR_SPIN_SPIN, [0, 1])
    s.close()
    with pytest.raises(pkg.SGSError) as e:
        pkg.Solver().admit(pkg.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, None, 0.05, shard=(2, 2))
    assert e.value.status == 1
