"""Host logic of the pair-sharded step (CPU): the partition of the pairs and the
two sums over ranks, driven by paper_2105_01088_gb300.sharded on two and three
gloo ranks (ranks without pairs included), with a stand-in backend that
evaluates each stage's share with the oracle.  Summed over the ranks, the
shares must give the single-rank oracle step: energies to 1e-12 relative and
the states to 1e-10."""
import os
import socket

import numpy as np
import pytest

import sgs_inputs as inp
from oracle import sgs_oracle as orc
from paper_2105_01088_gb300.sharded import ShardedStep, local_pairs, own_states, pair_list

torch = pytest.importorskip("torch")


class OracleShard:
    """Stage shares of one rank evaluated with the oracle (the three stage calls of
    the library, with the same layouts: [G | h] as complex (re, im) pairs, dGamma
    as [M][n][n])."""

    def __init__(self, model, gammas, rank, world, dtau, cmode=0):
        self.model, self.g = model, [np.array(x) for x in gammas]
        self.rank, self.world, self.dtau, self.cmode = rank, world, dtau, cmode
        self.M = len(gammas)

    def pairs(self):
        M = self.M
        G = np.zeros((M, M), complex)
        h = np.zeros((M, M), complex)
        for a, b in local_pairs(M, self.rank, self.world):
            G[a, b], h[b, a] = orc.pair_elements(self.model, self.g, a, b)
            G[b, a], h[a, b] = np.conj(G[a, b]), np.conj(h[b, a])
        for mu in own_states(M, self.rank, self.world):
            G[mu, mu] = 1.0
            h[mu, mu] = orc.wick_energy_density(self.model, self.g[mu])
        return torch.from_numpy(np.stack([G, h]).view(np.float64).ravel().copy())

    def eom(self, gh):
        M = self.M
        G, h = gh.numpy().view(np.complex128).reshape(2, M, M)
        E, lam = orc.solve_amplitudes(G, h)
        mine = set(local_pairs(M, self.rank, self.world))
        own = set(own_states(M, self.rank, self.world))

        def betas(mu):
            return [b for b in range(M) if (b == mu and mu in own) or (b != mu and (min(mu, b), max(mu, b)) in mine)]

        dG = orc.eom(self.model, self.g, G, h, E, lam, self.cmode, betas=betas)
        return E, torch.from_numpy(np.stack(dG).ravel().copy())

    def update(self, dg):
        n = self.model.n
        dG = dg.numpy().reshape(self.M, n, n)
        self.g = [orc.purify(orc.orthogonal_step(g, d, self.dtau)) for g, d in zip(self.g, dG)]


def _case(M=5):
    p = inp.AndersonParams(n_bath=4, U=2.0, eps_d=-1.0, V=0.5)           # n = 20
    rng = np.random.default_rng(31)
    g = inp.clustered_pure_gammas(p.n_modes, M, rng, 1, spread=1.0)
    return p, g


def _worker(rank, world, port, out_dir, n_steps, M=5):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, g = _case(M)
        model = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V)
        backend = OracleShard(model, g, rank, world, 0.05)
        E = ShardedStep(backend).step(n_steps)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), E=E, g=np.stack(backend.g))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_every_pair_once():
    for M in (1, 2, 5, 32):
        for world in (1, 2, 3, 8):
            got = sorted(ab for r in range(world) for ab in local_pairs(M, r, world))
            assert got == pair_list(M)
            assert sorted(mu for r in range(world) for mu in own_states(M, r, world)) == list(range(M))
            sizes = [len(local_pairs(M, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1             # balanced


@pytest.mark.parametrize("world,M", [(2, 5), (3, 5), (3, 2)])
def test_gloo_ranks_equal_the_single_rank_step(tmp_path, world, M):
    """Two ranks; three ranks with shares of 4, 3 and 3 pairs; and three ranks for two states,
    where ranks 1 and 2 hold no pair and rank 2 no state of its own (its shares are zero)."""
    import torch.multiprocessing as mp
    n_steps = 2
    sizes = [len(local_pairs(M, r, world)) for r in range(world)]
    assert sizes == {(2, 5): [5, 5], (3, 5): [4, 3, 3], (3, 2): [1, 0, 0]}[(world, M)]
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path), n_steps, M), nprocs=world, join=True)
    p, g = _case(M)
    model = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V)
    Eo, _, go = orc.run(model, list(g), 0.05, n_steps)
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    for r in res:
        assert np.all(np.abs(r["E"] - Eo) <= 1e-12 * np.abs(Eo))
        assert np.abs(r["g"] - np.stack(go)).max() <= 1e-10
    # and the ranks agree with each other exactly (the same sums, the same update)
    for r in res[1:]:
        assert np.array_equal(res[0]["g"], r["g"]) and np.array_equal(res[0]["E"], r["E"])
