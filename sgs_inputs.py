"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  Holds no arithmetic of the SGS method itself: it draws model
parameters, random pure covariance matrices and random amplitudes.

Random pure states: Gamma = O J O^T with O Haar-distributed on O(2N) (QR of a
standard normal matrix with the signs of diag(R) folded into Q), one column
flipped if needed so that det O (= Pf Gamma, the fermion parity) equals the
requested parity.  Amplitudes: lambda_mu = exp(i theta), theta ~ U[0, 2 pi).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def vacuum_gamma(n_modes: int) -> np.ndarray:
    n = 2 * n_modes
    J = np.zeros((n, n))
    for m in range(n_modes):
        J[2 * m, 2 * m + 1] = 1.0
        J[2 * m + 1, 2 * m] = -1.0
    return J


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(R))


def random_pure_gamma(n_modes: int, rng: np.random.Generator, parity: int = 1) -> np.ndarray:
    n = 2 * n_modes
    O = haar_orthogonal(n, rng)
    if np.linalg.det(O) * parity < 0:
        O[:, 0] = -O[:, 0]
    G = O @ vacuum_gamma(n_modes) @ O.T
    return 0.5 * (G - G.T)


def clustered_pure_gammas(n_modes: int, M: int, rng: np.random.Generator, parity: int = 1,
                          spread: float = 0.5) -> np.ndarray:
    """M pure states Gamma_mu = O_mu Gamma_0 O_mu^T around one Haar-random
    Gamma_0, with O_mu = exp(K_mu), K_mu antisymmetric with N(0, s^2) entries
    and s = spread / (2 n_modes): mutual overlaps of order one, as between
    the states of an ansatz grown by small rotations of existing states."""
    import scipy.linalg
    n = 2 * n_modes
    base = random_pure_gamma(n_modes, rng, parity)
    out = []
    for _ in range(M):
        K = rng.standard_normal((n, n)) * (spread / n)
        K = K - K.T
        O = scipy.linalg.expm(K)
        G = O @ base @ O.T
        out.append(0.5 * (G - G.T))
    return np.ascontiguousarray(np.stack(out))


# ---------------------------------------------------------------------------
# Counter-based seeded states (the same definition the library uses when it
# generates initial states itself): Philox4x32-10 (Salmon et al., SC11), key =
# the 64-bit seed; state mu's standard-normal matrix entries 2j, 2j+1 from
# counter (j, mu, 0, 0) by Box-Muller on the first two words; the phase of
# lambda_mu from counter (0, mu, 1, 0); O Haar from QR with sign(diag R).

_PHILOX_M0, _PHILOX_M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_PHILOX_W0, _PHILOX_W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32(counters: np.ndarray, seed: int) -> np.ndarray:
    """Philox4x32-10 of each row of counters ([k, 4] integers < 2^32); returns [k, 4] uint64."""
    x = [np.asarray(counters[:, i], dtype=np.uint64) for i in range(4)]
    k0, k1 = np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = (k0 + _PHILOX_W0) & _MASK32
            k1 = (k1 + _PHILOX_W1) & _MASK32
        p0 = _PHILOX_M0 * x[0]
        p1 = _PHILOX_M1 * x[2]
        x = [(p1 >> np.uint64(32)) ^ x[1] ^ k0, p1 & _MASK32, (p0 >> np.uint64(32)) ^ x[3] ^ k1, p0 & _MASK32]
    return np.stack(x, 1)


def seeded_state(n_modes: int, mu: int, seed: int, parity: int = 1):
    n = 2 * n_modes
    j = np.arange(n * n // 2, dtype=np.uint64)
    ctr = np.stack([j, np.full_like(j, mu), np.zeros_like(j), np.zeros_like(j)], 1)
    x = philox4x32(ctr, seed)
    u1 = (x[:, 0].astype(np.float64) + 1.0) / 4294967296.0
    u2 = x[:, 1].astype(np.float64) / 4294967296.0
    r = np.sqrt(-2.0 * np.log(u1))
    Z = np.empty(n * n)
    Z[0::2] = r * np.cos(2.0 * np.pi * u2)
    Z[1::2] = r * np.sin(2.0 * np.pi * u2)
    Q, R = np.linalg.qr(Z.reshape(n, n))
    O = Q * np.sign(np.diag(R))
    if np.sign(np.linalg.det(O)) != parity:
        O[:, 0] = -O[:, 0]
    g = O @ vacuum_gamma(n_modes) @ O.T
    x = philox4x32(np.array([[0, mu, 1, 0]], dtype=np.uint64), seed)
    th = 2.0 * np.pi * float(x[0, 0]) / 4294967296.0
    return 0.5 * (g - g.T), np.exp(1j * th)


def seeded_states(n_modes: int, M: int, seed: int, parity: int = 1):
    out = [seeded_state(n_modes, mu, seed, parity) for mu in range(M)]
    return np.stack([g for g, _ in out]), np.array([l for _, l in out])


def random_generator(n: int, norm: float, rng: np.random.Generator) -> np.ndarray:
    """A random antisymmetric n x n matrix K with ||K||_F = norm (exactly
    antisymmetric: K = X - X^T, scaled), so that exp(K) is a random special
    orthogonal matrix with ||exp(K) - 1||_F ~ norm."""
    X = rng.standard_normal((n, n))
    K = X - X.T
    K *= norm / np.linalg.norm(K)
    return 0.5 * (K - K.T)


def random_amplitudes(M: int, rng: np.random.Generator) -> np.ndarray:
    return np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=M))


@dataclass
class AndersonParams:
    """Anderson impurity with ``n_channels`` open bath chains (Sec. IV model;
    two channels for the two-channel impurity workload)."""
    n_bath: int
    U: float
    eps_d: float
    V: float
    t: float = 1.0
    mu: float = 0.0
    n_channels: int = 1

    @property
    def n_sites(self) -> int:
        return 1 + self.n_channels * self.n_bath

    @property
    def n_modes(self) -> int:
        return 2 * self.n_sites


@dataclass
class Workload:
    name: str
    model: AndersonParams
    rank: int
    dtau: float
    n_steps: int
    seed: int
    parity: int = 1
    extra: dict = field(default_factory=dict)


def initial_state(n_modes: int, rank: int, seed: int, parity: int = 1):
    """(gammas [rank, 2N, 2N] float64, lambdas [rank] complex128) from one seed."""
    rng = np.random.default_rng(seed)
    gammas = np.stack([random_pure_gamma(n_modes, rng, parity) for _ in range(rank)])
    lam = random_amplitudes(rank, rng)
    return np.ascontiguousarray(gammas), lam


# Workloads: a small plain-FP64 case (16 sites, N=32 modes, M=4), the
# throughput case (128 sites, N=256, M=32), the two-channel case (201 sites,
# N=402, M=64), and the batched uneven case (256 instances).
SMALL = Workload("anderson_L16_M4", AndersonParams(n_bath=15, U=2.0, eps_d=-1.0, V=0.5), rank=4,
                 dtau=0.05, n_steps=200, seed=1)
LARGE = Workload("anderson_L128_M32", AndersonParams(n_bath=127, U=4.0, eps_d=-2.0, V=0.5), rank=32,
                 dtau=0.05, n_steps=500, seed=2)
TWO_CHANNEL = Workload("two_channel_L201_M64",
                       AndersonParams(n_bath=100, U=8.0, eps_d=-4.0, V=0.6, n_channels=2), rank=64,
                       dtau=0.05, n_steps=1000, seed=3, parity=-1)
# the system of Sec. IV A's energy extrapolation: L = 500 sites (impurity + 499 bath sites), U = t = 1,
# U / Gamma = 5 with Gamma = t'^2 / t, mu = 0, eps_d = -U/2; rank 16, the largest rank the paper reports there
SIAM_L500 = Workload("siam_L500_M16", AndersonParams(n_bath=499, U=1.0, eps_d=-0.5, V=0.2 ** 0.5), rank=16,
                     dtau=0.05, n_steps=0, seed=5)


def batched_workloads(n_instances: int = 256, seed: int = 4, dtau: float = 0.05, n_bath=(16, 256),
                      ranks=(8, 16, 32)):
    """Uneven instances: bath length L ~ U{n_bath} per spin (default 16..256),
    rank M from ``ranks`` (default {8, 16, 32}), U ~ U[0, 8], eps_d = -U/2,
    V ~ U[0.2, 1.0]."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_instances):
        L = int(rng.integers(n_bath[0], n_bath[1] + 1))
        M = int(rng.choice(list(ranks)))
        U = float(rng.uniform(0.0, 8.0))
        V = float(rng.uniform(0.2, 1.0))
        # L bath sites plus the impurity; half filling puts L + 1 electrons
        # in the particle-hole symmetric ground state, hence its parity
        out.append(Workload(f"batched_{i}", AndersonParams(n_bath=L, U=U, eps_d=-U / 2, V=V), rank=M,
                            dtau=dtau, n_steps=1, seed=int(rng.integers(1 << 31)),
                            parity=1 if (L + 1) % 2 == 0 else -1))
    return out


def serving_requests(rate: float, n_requests: int, seed: int = 5, n_bath=(8, 40), ranks=(4, 8)):
    """A seeded Poisson stream of impurity solves: exponential inter-arrival times
    at ``rate`` per second; per request an Anderson model with bath length
    L ~ U{n_bath}, rank M from ``ranks``, U ~ U[0, 8], eps_d = -U/2, V ~ U[0.2, 1.0],
    and random pure initial states.  Returns [(arrival, AndersonParams, M, seed, parity)]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        L = int(rng.integers(n_bath[0], n_bath[1] + 1))
        M = int(rng.choice(ranks))
        U = float(rng.uniform(0.0, 8.0))
        V = float(rng.uniform(0.2, 1.0))
        out.append((t, AndersonParams(n_bath=L, U=U, eps_d=-U / 2, V=V), M, int(rng.integers(1 << 31)),
                    1 if (L + 1) % 2 == 0 else -1))
    return out
