"""GB300 (sm_103a) imaginary-time step of the superposition-of-Gaussian-states
variational method (Boutin & Bauer, arXiv:2105.01088).

Thin Python binding over the C ABI of include/sgs.h (libsgs.so, built in tree
by ``paper_2105_01088_gb300.build``).  Every step of the method runs in the
library's CUDA kernels; this module only marshals arguments.  PyTorch, when
present with a GPU, provides the device memory (its caching allocator) and
the CUDA stream.  The first call raises ImportError if the library has not
been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgs.so")

SGS_FP64, SGS_MIXED_TF32, SGS_MIXED_BF16, SGS_FP32_3XTF32 = 0, 1, 2, 3
FP64_EMULATED, FP64_FMA = 0, 1          # sgs_fp64_path: arithmetic of the FP64 products
SGS_C_INVERSE, SGS_C_PHASE = 0, 1
SGS_INTEGRATOR_EXP, SGS_INTEGRATOR_EULER = 0, 1
SGS_CORR_SPIN_SPIN, SGS_CORR_TWO_CHANNEL_K, SGS_CORR_RENYI2 = 0, 1, 2
STATUS = {0: "SGS_OK", 1: "SGS_EINVAL", 2: "SGS_ENOMEM", 3: "SGS_ESINGULAR", 4: "SGS_ENOTCONV",
          5: "SGS_ETIMEOUT", 6: "SGS_ECUDA"}


class SGSError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


class _Model(ctypes.Structure):
    _fields_ = [("n_modes", ctypes.c_int), ("A", ctypes.POINTER(ctypes.c_double)), ("n_quartic", ctypes.c_int),
                ("quartic_idx", ctypes.POINTER(ctypes.c_int)), ("quartic_val", ctypes.POINTER(ctypes.c_double)),
                ("e_const", ctypes.c_double), ("n_higher", ctypes.c_int),
                ("higher_len", ctypes.POINTER(ctypes.c_int)), ("higher_idx", ctypes.POINTER(ctypes.c_int)),
                ("higher_val", ctypes.POINTER(ctypes.c_double))]


class _Options(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int), ("dtau", ctypes.c_double), ("precision", ctypes.c_int),
                ("cmode", ctypes.c_int), ("parity", ctypes.c_int), ("gamma0", ctypes.POINTER(ctypes.c_double)),
                ("lambda0", ctypes.POINTER(ctypes.c_double)), ("stream", ctypes.c_void_p),
                ("integrator", ctypes.c_int), ("seed", ctypes.c_ulonglong), ("fp64_path", ctypes.c_int),
                ("emulation_scratch", ctypes.c_size_t), ("shard_rank", ctypes.c_int), ("shard_world", ctypes.c_int),
                ("pair_chunk", ctypes.c_int)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_ctxp = ctypes.c_void_p

# exported symbols and their signatures (must match include/sgs.h)
SIGNATURES = {
    "sgs_init": (ctypes.c_int, [ctypes.POINTER(_Model), ctypes.POINTER(_Options), ctypes.c_int,
                                ctypes.POINTER(ctypes.c_void_p)]),
    "sgs_step": (ctypes.c_int, [_ctxp, ctypes.c_int, _dp]),
    "sgs_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]),
    "sgs_admit": (ctypes.c_int, [_ctxp, ctypes.POINTER(_Model), ctypes.POINTER(_Options), ctypes.POINTER(ctypes.c_int)]),
    "sgs_retire": (ctypes.c_int, [_ctxp, ctypes.c_int]),
    "sgs_bytes_in_use": (ctypes.c_size_t, [_ctxp]),
    "sgs_add_state": (ctypes.c_int, [_ctxp, ctypes.c_int, _dp, ctypes.c_int]),
    "sgs_set_autotune": (ctypes.c_int, [_ctxp, ctypes.c_int]),
    "sgs_failed_instance": (ctypes.c_int, [_ctxp]),
    "sgs_failed_instances": (ctypes.c_int, [_ctxp, _ip, ctypes.c_int]),
    "sgs_health": (ctypes.c_int, [_ctxp, ctypes.c_int, _dp]),
    "sgs_seeded_states": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_int, _dp, _dp]),
    "sgs_get_tuning": (ctypes.c_int, [_ctxp, ctypes.c_int, _ip, _ip, _ip]),
    "sgs_set_panel_widths": (ctypes.c_int, [_ctxp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "sgs_set_graphs": (ctypes.c_int, [_ctxp, ctypes.c_int]),
    "sgs_energy": (ctypes.c_int, [_ctxp, _dp]),
    "sgs_shard_pairs": (ctypes.c_int, [_ctxp, ctypes.c_int, ctypes.c_void_p]),
    "sgs_shard_eom": (ctypes.c_int, [_ctxp, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, _dp]),
    "sgs_shard_update": (ctypes.c_int, [_ctxp, ctypes.c_int, ctypes.c_void_p]),
    "sgs_correlator": (ctypes.c_int, [_ctxp, ctypes.c_int, ctypes.c_int, _ip, ctypes.c_int, _dp]),
    "sgs_variance": (ctypes.c_int, [_ctxp, ctypes.c_int, _dp, _dp]),
    "sgs_free": (None, [_ctxp]),
    "sgs_last_error": (ctypes.c_char_p, [_ctxp]),
    "sgs_get_state": (ctypes.c_int, [_ctxp, ctypes.c_int, _dp, _dp]),
    "sgs_set_state": (ctypes.c_int, [_ctxp, ctypes.c_int, _dp, _dp]),
    "sgs_get_pair_matrices": (ctypes.c_int, [_ctxp, ctypes.c_int, _dp, _dp]),
    "sgs_get_derivative": (ctypes.c_int, [_ctxp, ctypes.c_int, _dp]),
    "sgs_set_allocator": (None, [_ALLOC_FN, _FREE_FN, ctypes.c_void_p]),
    "sgs_build_anderson": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _ip, _dp, _dp]),
    "sgs_build_2ck": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _ip, _dp, _dp]),
    "sgs_set_profiling": (ctypes.c_int, [_ctxp, ctypes.c_int]),
    "sgs_get_profile": (ctypes.c_int, [_ctxp, _dp, _dp, _dp, ctypes.POINTER(ctypes.c_longlong), _dp]),
    "sgs_probe_peak": (ctypes.c_int, [ctypes.c_int, _dp]),
    "sgs_kernel_smem_limits": (ctypes.c_int, [ctypes.c_int, _ip, _ip]),
    "sgs_probe_wait": (ctypes.c_int, [ctypes.c_ulonglong, _dp]),
    "sgs_kernel_inverse": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]),
    "sgs_kernel_pfaffian": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]),
    "sgs_kernel_gemm": (ctypes.c_int, [_dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, _dp]),
    "sgs_kernel_gemm_tc": (ctypes.c_int, [_dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, _dp]),
    "sgs_kernel_inverse_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_void_p]),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2105_01088_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


class _LazyLibrary:
    """Loads libsgs.so on first use (so that ``paper_2105_01088_gb300.build``
    can run before the library exists); raises ImportError if it is missing."""

    _cdll = None

    def __getattr__(self, name):
        if _LazyLibrary._cdll is None:
            _LazyLibrary._cdll = load_library()
        return getattr(_LazyLibrary._cdll, name)


_lib = _LazyLibrary()


def _ptr(a, kind=_dp):
    return a.ctypes.data_as(kind) if a is not None else None


# ------------------------------------------------------------ device memory via PyTorch
_torch_hooks = None


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching
    allocator (call once, before creating solvers)."""
    global _torch_hooks
    if _torch_hooks is not None:
        return
    import torch

    def _alloc(nbytes, stream, user):
        try:
            s = stream if stream else torch.cuda.current_stream().cuda_stream
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), s)
        except Exception:
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)

    _torch_hooks = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _lib.sgs_set_allocator(_torch_hooks[0], _torch_hooks[1], None)


# ------------------------------------------------------------ model builder

class MajoranaModel:
    """Model in the library's input form: A (n x n), quartic monomials
    (idx [q, 4], val [q]), the constant e_const (Sec. II A) and terms of six or
    eight Majoranas, ``higher`` = [(indices, v)] for v i^(r mod 2) c_s1 ... c_s2r."""

    def __init__(self, A, quartic_idx, quartic_val, e_const, higher=()):
        self.A = np.ascontiguousarray(A, dtype=np.float64)
        self.quartic_idx = np.ascontiguousarray(np.asarray(quartic_idx, dtype=np.int32).reshape(-1, 4))
        self.quartic_val = np.ascontiguousarray(quartic_val, dtype=np.float64).reshape(-1)
        self.e_const = float(e_const)
        self.higher = [(tuple(int(x) for x in idx), float(v)) for idx, v in higher]
        self.n = self.A.shape[0]
        self.n_modes = self.n // 2

    def with_higher(self, higher):
        """The same model plus terms of six or eight Majoranas."""
        return MajoranaModel(self.A, self.quartic_idx, self.quartic_val, self.e_const, list(self.higher) + list(higher))

    def _struct(self):
        """The sgs_model of this model and the arrays it points into (kept alive by the caller)."""
        hl = np.ascontiguousarray([len(i) for i, _ in self.higher], dtype=np.int32)
        hi = np.ascontiguousarray([x for i, _ in self.higher for x in i], dtype=np.int32)
        hv = np.ascontiguousarray([v for _, v in self.higher], dtype=np.float64)
        keep = (hl, hi, hv)
        nh = len(self.higher)
        return _Model(self.n_modes, _ptr(self.A), len(self.quartic_val), _ptr(self.quartic_idx, _ip),
                      _ptr(self.quartic_val), self.e_const, nh, _ptr(hl, _ip) if nh else None,
                      _ptr(hi, _ip) if nh else None, _ptr(hv) if nh else None), keep


def build_anderson(n_bath, U, eps_d, V, t=1.0, mu=0.0, n_channels=1) -> MajoranaModel:
    n_sites = 1 + n_channels * n_bath
    n = 4 * n_sites
    A = np.zeros((n, n))
    qi = np.zeros(4, dtype=np.int32)
    qv = np.zeros(1)
    ec = np.zeros(1)
    nm = _lib.sgs_build_anderson(n_bath, n_channels, U, eps_d, V, t, mu, _ptr(A), _ptr(qi, _ip), _ptr(qv), _ptr(ec))
    if nm < 0:
        raise SGSError(1, "bad Anderson parameters")
    return MajoranaModel(A, qi, qv, ec[0])


def build_2ck(L, J, t=0.5) -> MajoranaModel:
    """Lattice two-channel Kondo model of Sec. V (2L sites)."""
    n = 8 * L
    A = np.zeros((n, n))
    qi = np.zeros(24 * 4, dtype=np.int32)
    qv = np.zeros(24)
    ec = np.zeros(1)
    nm = _lib.sgs_build_2ck(L, J, t, _ptr(A), _ptr(qi, _ip), _ptr(qv), _ptr(ec))
    if nm < 0:
        raise SGSError(1, "bad two-channel Kondo parameters")
    return MajoranaModel(A, qi, qv, ec[0])


def seeded_states(n_modes, rank, seed, parity=1):
    """The states sgs_admit generates without gamma0: (gamma [rank, 2N, 2N], lambda [rank])."""
    n = 2 * n_modes
    g = np.zeros((rank, n, n))
    lam = np.zeros((rank, 2))
    st = _lib.sgs_seeded_states(n_modes, rank, int(seed), parity, _ptr(g), _ptr(lam))
    if st != 0:
        raise SGSError(st, "bad arguments")
    return g, lam[:, 0] + 1j * lam[:, 1]


# ------------------------------------------------------------ solver

def _check_slot_args(model, gamma0, parity, rank=None):
    if gamma0 is None:
        M = rank
        if M is None:
            raise SGSError(1, "without gamma0 the rank must be given")
    else:
        g = np.asarray(gamma0)
        if g.ndim != 3 or g.shape[1:] != (model.n, model.n):
            raise SGSError(1, f"gamma0 has shape {g.shape}, expected (M, {model.n}, {model.n})")
        M = g.shape[0]
    if not 1 <= M <= 64:
        raise SGSError(1, f"rank {M} outside 1..64")
    if parity not in (1, -1):
        raise SGSError(1, f"parity {parity} is not +-1")


class Solver:
    """A context of independent SGS problems (slots) resident on the GPU.

    models: MajoranaModel or list; gamma0: [M, n, n] or list; lambda0: [M]
    complex or None.  stream: a CUDA stream handle (int), a torch stream, or
    None (a stream of the library's own).  hbm_budget: bytes the live slots may
    hold (0: no budget).  fp64_path: FP64_EMULATED (default) or FP64_FMA for the
    FP64 products of every slot this constructor admits; emulation_scratch:
    slice scratch per slot (bytes, 0: the library's default).  Slots can be
    added (admit) and released (retire) while others are live: continuous
    batching."""

    def __init__(self, models=(), gamma0=(), lambda0=None, dtau=0.05, precision=SGS_FP64, cmode=SGS_C_INVERSE,
                 parity=1, stream=None, hbm_budget=0, integrator=SGS_INTEGRATOR_EXP, autotune=False,
                 fp64_path=FP64_EMULATED, emulation_scratch=0, pair_chunk=0):
        if isinstance(models, MajoranaModel):
            models, gamma0, lambda0 = [models], [gamma0], [lambda0]
        models = list(models)
        k = len(models)

        def per(x):
            return list(x) if isinstance(x, (list, tuple)) else [x] * k

        if lambda0 is None:
            lambda0 = [None] * k
        for m, g, pa in zip(models, gamma0, per(parity)):
            _check_slot_args(m, g, pa)          # before any CUDA call
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._stream = stream
        ctx = ctypes.c_void_p()
        st = _lib.sgs_create(ctypes.c_void_p(stream) if stream else None, int(hbm_budget), ctypes.byref(ctx))
        if st != 0:
            raise SGSError(st, "sgs_create failed")
        self._ctx = ctx
        if autotune:
            _lib.sgs_set_autotune(ctx, 1)
        self.shapes = []
        self.live = []
        self._keep = {}
        self.fp64_path, self.emulation_scratch = int(fp64_path), int(emulation_scratch)
        self.pair_chunk = int(pair_chunk)
        for i, m, g, l0, dt, pr, cm, pa, it in zip(range(k), models, gamma0, lambda0, per(dtau), per(precision),
                                                   per(cmode), per(parity), per(integrator)):
            try:
                self.admit(m, g, l0, dt, pr, cm, pa, it)
            except SGSError:
                self.close()
                raise

    @property
    def n_instances(self):
        return len(self.shapes)

    def admit(self, model, gamma0, lambda0=None, dtau=0.05, precision=SGS_FP64, cmode=SGS_C_INVERSE, parity=1,
              integrator=SGS_INTEGRATOR_EXP, rank=None, seed=0, fp64_path=None, emulation_scratch=None,
              shard=(0, 1), pair_chunk=None):
        """Add one problem; returns its slot.  gamma0 None: seeded random states of
        the given rank, generated by the library.  fp64_path / emulation_scratch:
        None takes the solver's.  shard = (rank, world): this rank's share of a
        pair-sharded step (sharded.py).  pair_chunk: per-pair buffers for this many
        pairs, the step running the pairs in chunks (bounded memory; None takes the
        solver's, 0 all pairs).  Raises SGSError(SGS_ENOMEM) if it does not fit the
        HBM budget (nothing is allocated then)."""
        _check_slot_args(model, gamma0, parity, rank)
        g = None if gamma0 is None else np.ascontiguousarray(gamma0, dtype=np.float64)
        M = rank if g is None else g.shape[0]
        lam = None
        if lambda0 is not None:
            lam = np.ascontiguousarray(np.stack([np.real(lambda0), np.imag(lambda0)], -1), dtype=np.float64)
        mod, _keep = model._struct()
        path = self.fp64_path if fp64_path is None else int(fp64_path)
        scratch = self.emulation_scratch if emulation_scratch is None else int(emulation_scratch)
        chunk = self.pair_chunk if pair_chunk is None else int(pair_chunk)
        opt = _Options(M, dtau, precision, cmode, parity, _ptr(g), _ptr(lam), None, integrator, int(seed), path,
                       scratch, int(shard[0]), int(shard[1]), chunk)
        slot = ctypes.c_int(-1)
        st = _lib.sgs_admit(self._ctx, ctypes.byref(mod), ctypes.byref(opt), ctypes.byref(slot))
        if st != 0:
            raise SGSError(st, (_lib.sgs_last_error(self._ctx) or b"").decode())
        self.shapes.append((M, model.n))
        self.live.append(True)
        return slot.value

    def retire(self, slot):
        self._check(_lib.sgs_retire(self._ctx, slot))
        self.live[slot] = False

    def bytes_in_use(self):
        return int(_lib.sgs_bytes_in_use(self._ctx))

    def health(self, instance=0):
        """{purity_residual, nonfinite, gram_eig_ratio, energy} of the current states."""
        out = np.zeros(4)
        self._check(_lib.sgs_health(self._ctx, instance, _ptr(out)))
        return {"purity_residual": out[0], "nonfinite": int(out[1]), "gram_eig_ratio": out[2], "energy": out[3]}

    def failed_instance(self):
        """First slot whose device-side error ended the last call (-1: none)."""
        return int(_lib.sgs_failed_instance(self._ctx))

    def failed_instances(self):
        """Every slot whose device-side error ended the last call."""
        n = int(_lib.sgs_failed_instances(self._ctx, None, 0))
        out = np.zeros(max(n, 1), dtype=np.int32)
        _lib.sgs_failed_instances(self._ctx, _ptr(out, _ip), n)
        return [int(x) for x in out[:n]]

    def tuning(self, slot=0):
        """(Gauss-Jordan panel width, Pfaffian panel width, source) of a slot;
        source -1 not tuned, 0 timed, 1 cached."""
        v = [ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)]
        self._check(_lib.sgs_get_tuning(self._ctx, slot, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def set_panel_widths(self, gj_width, pf_width, slot=0):
        """Fix a slot's panel widths (each one of the autotuner's candidates, within
        the slot's scratch)."""
        self._check(_lib.sgs_set_panel_widths(self._ctx, slot, int(gj_width), int(pf_width)))

    def add_state(self, K, src=-1, slot=0):
        """Rank growth (Sec. III C): append Q Gamma_src Q^T, Q = exp(K), to a
        slot (K antisymmetric [n, n]; src -1: the state of largest amplitude)."""
        M, n = self.shapes[slot]
        k = np.ascontiguousarray(K, dtype=np.float64)
        if k.shape != (n, n):
            raise SGSError(1, f"K has shape {k.shape}, expected ({n}, {n})")
        self._check(_lib.sgs_add_state(self._ctx, slot, _ptr(k), int(src)))
        self.shapes[slot] = (M + 1, n)

    def _check(self, st):
        if st != 0:
            raise SGSError(st, (_lib.sgs_last_error(self._ctx) or b"").decode())

    def step(self, n_steps=1) -> np.ndarray:
        """Advance every live slot; returns energies [n_slots, n_steps] (NaN rows
        for retired slots).  On a device-side failure of some slots the SGSError
        carries ``energies`` (NaN rows for the failed ones) and ``failed`` (their
        slots)."""
        E = np.full((self.n_instances, n_steps), np.nan)
        st = _lib.sgs_step(self._ctx, n_steps, _ptr(E))
        if st != 0:
            err = SGSError(st, (_lib.sgs_last_error(self._ctx) or b"").decode())
            err.energies = E
            err.failed = self.failed_instances()
            raise err
        return E

    def shard_pairs(self, gh_ptr, slot=0):
        """Stage 1 of a pair-sharded step: this rank's share of [G | h] into gh_ptr."""
        self._check(_lib.sgs_shard_pairs(self._ctx, slot, ctypes.c_void_p(gh_ptr)))

    def shard_eom(self, gh_ptr, dgamma_ptr, slot=0):
        """Stage 2: amplitudes from the summed gh, this rank's share of dGamma/ds into
        dgamma_ptr; returns the energy."""
        e = np.zeros(1)
        self._check(_lib.sgs_shard_eom(self._ctx, slot, ctypes.c_void_p(gh_ptr), ctypes.c_void_p(dgamma_ptr),
                                       _ptr(e)))
        return float(e[0])

    def shard_update(self, dgamma_ptr, slot=0):
        """Stage 3: the update of every state from the summed dGamma/ds."""
        self._check(_lib.sgs_shard_update(self._ctx, slot, ctypes.c_void_p(dgamma_ptr)))

    def set_graphs(self, enable=True):
        """Replay a captured CUDA graph of one step (default on)."""
        self._check(_lib.sgs_set_graphs(self._ctx, 1 if enable else 0))

    def energy(self) -> np.ndarray:
        E = np.full(self.n_instances, np.nan)
        self._check(_lib.sgs_energy(self._ctx, _ptr(E)))
        return E

    def correlator(self, kind, sites, instance=0) -> np.ndarray:
        s = np.ascontiguousarray(sites, dtype=np.int32)
        out = np.zeros(len(s))
        self._check(_lib.sgs_correlator(self._ctx, instance, kind, _ptr(s, _ip), len(s), _ptr(out)))
        return out

    def variance(self, instance=0):
        """(E, delta_H^2) of the current states (Eq. residual)."""
        e = np.zeros(1)
        v = np.zeros(1)
        self._check(_lib.sgs_variance(self._ctx, instance, _ptr(e), _ptr(v)))
        return float(e[0]), float(v[0])

    def get_state(self, instance=0, out=None):
        """(gamma [M, n, n], lambda [M]); ``out`` may be a C-contiguous float64
        [M, n, n] buffer (e.g. pinned host memory) to receive gamma."""
        M, n = self.shapes[instance]
        g = np.zeros((M, n, n)) if out is None else out
        if g.shape != (M, n, n) or g.dtype != np.float64 or not g.flags.c_contiguous:
            raise SGSError(1, "out must be a C-contiguous float64 array of shape (M, n, n)")
        lam = np.zeros((M, 2))
        self._check(_lib.sgs_get_state(self._ctx, instance, _ptr(g), _ptr(lam)))
        return g, lam[:, 0] + 1j * lam[:, 1]

    def set_state(self, gamma, lam=None, instance=0):
        g = np.ascontiguousarray(gamma, dtype=np.float64)
        l2 = None if lam is None else np.ascontiguousarray(np.stack([np.real(lam), np.imag(lam)], -1))
        self._check(_lib.sgs_set_state(self._ctx, instance, _ptr(g), _ptr(l2)))

    def pair_matrices(self, instance=0):
        M, _ = self.shapes[instance]
        G = np.zeros((M, M, 2))
        h = np.zeros((M, M, 2))
        self._check(_lib.sgs_get_pair_matrices(self._ctx, instance, _ptr(G), _ptr(h)))
        return G[..., 0] + 1j * G[..., 1], h[..., 0] + 1j * h[..., 1]

    def derivative(self, instance=0):
        M, n = self.shapes[instance]
        d = np.zeros((M, n, n))
        self._check(_lib.sgs_get_derivative(self._ctx, instance, _ptr(d)))
        return d

    STAGES = ("pair_inverse", "pair_delta", "phase_pfaffian", "amplitudes", "eom_w", "eom_v", "eom_x",
              "eom_assembly", "update")

    def set_profiling(self, enable=True):
        self._check(_lib.sgs_set_profiling(self._ctx, 1 if enable else 0))

    def profile(self):
        """({stage: (ms, flops, bytes)}, launches, (gemm_f64 ms, flops, launches))"""
        k = len(self.STAGES)
        ms, fl, by = np.zeros(k), np.zeros(k), np.zeros(k)
        gk = np.zeros(3)
        nl = ctypes.c_longlong(0)
        self._check(_lib.sgs_get_profile(self._ctx, _ptr(ms), _ptr(fl), _ptr(by), ctypes.byref(nl), _ptr(gk)))
        return {s: (ms[i], fl[i], by[i]) for i, s in enumerate(self.STAGES)}, nl.value, tuple(gk)

    def close(self):
        if getattr(self, "_ctx", None):
            _lib.sgs_free(self._ctx)
            self._ctx = None

    def __del__(self):
        self.close()


# ------------------------------------------------------------ building blocks

def probe_wait(limit_ns):
    """Run the bounded device wait on a flag nothing sets; returns (status, device ms)."""
    ms = np.zeros(1)
    st = _lib.sgs_probe_wait(int(limit_ns), _ptr(ms))
    return int(st), float(ms[0])


def smem_limits():
    """[(dynamic shared-memory limit in force, opt-in maximum less static shared
    memory)] of the library's large-shared-memory kernels on the current device."""
    lim = np.zeros(9, dtype=np.int32)
    exp = np.zeros(9, dtype=np.int32)
    st = _lib.sgs_kernel_smem_limits(9, _ptr(lim, _ip), _ptr(exp, _ip))
    if st != 0:
        raise SGSError(st, "shared-memory limits")
    return list(zip(lim.tolist(), exp.tolist()))


def probe_peak(kind=0):
    """Measured TFLOP/s of the FP64 MMA (kind 0), FP64 FMA (kind 1), or both
    interleaved (kind 2)."""
    out = np.zeros(1)
    st = _lib.sgs_probe_peak(kind, _ptr(out))
    if st != 0:
        raise SGSError(st, "probe")
    return float(out[0])


def batched_inverse(S, fp64_path=FP64_EMULATED):
    S = np.ascontiguousarray(S, dtype=np.float64)
    b, n, _ = S.shape
    out = np.zeros_like(S)
    ld = np.zeros(b)
    st = _lib.sgs_kernel_inverse(_ptr(S), n, b, int(fp64_path), _ptr(out), _ptr(ld))
    if st != 0:
        raise SGSError(st, "batched inverse")
    return out, ld


def batched_inverse_static(S_ptr, inv_ptr, logabsdet_ptr, n, batch, stream=None):
    """Allocation-free batched inverse on caller-owned DEVICE buffers (raw
    pointers, e.g. ``tensor.data_ptr()``); see sgs_kernel_inverse_static."""
    st = _lib.sgs_kernel_inverse_static(ctypes.c_void_p(S_ptr), ctypes.c_void_p(inv_ptr),
                                        ctypes.c_void_p(logabsdet_ptr), n, batch,
                                        ctypes.c_void_p(stream) if stream else None)
    if st != 0:
        raise SGSError(st, "allocation-free batched inverse")


def batched_gemm_tc(A, B, kind=0):
    """batch C = A B on the tcgen05 tensor cores (kind 0 TF32, 1 BF16, 2 3xTF32)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    Bt = np.ascontiguousarray(np.swapaxes(np.asarray(B, dtype=np.float64), 1, 2))
    b, m, k = A.shape
    n = Bt.shape[1]
    C = np.zeros((b, m, n))
    st = _lib.sgs_kernel_gemm_tc(_ptr(A), _ptr(Bt), m, n, k, b, kind, _ptr(C))
    if st != 0:
        raise SGSError(st, "tensor-core gemm")
    return C


def batched_pfaffian(Y, fp64_path=FP64_EMULATED):
    Y = np.ascontiguousarray(Y, dtype=np.complex128)
    b, n, _ = Y.shape
    yv = Y.view(np.float64)
    ph = np.zeros((b, 2))
    la = np.zeros(b)
    st = _lib.sgs_kernel_pfaffian(_ptr(yv), n, b, int(fp64_path), _ptr(ph), _ptr(la))
    if st != 0:
        raise SGSError(st, "batched pfaffian")
    return ph[:, 0] + 1j * ph[:, 1], la


def batched_gemm(A, B, Cin=None, alpha=1.0, beta=0.0, diag=0.0, trans_a=False, trans_b=False, mode=0,
                 gj=(0, 1), C=None, b_antisym=False, fp64_path=FP64_EMULATED, emulation_scratch=0):
    """batch C = alpha op(A) op(B) + beta Cin + diag I through the library's FP64
    product (mode 0 full, 1 antisymmetric, 2 Gauss-Jordan update with panel
    columns gj = (k0, b) left unchanged).  C (optional) holds the output's initial
    values.  b_antisym declares B antisymmetric (the emulated path then slices its
    rows); emulation_scratch caps the slice scratch (bytes, 0: default)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    b = A.shape[0]
    m, k = (A.shape[2], A.shape[1]) if trans_a else (A.shape[1], A.shape[2])
    n = B.shape[1] if trans_b else B.shape[2]
    out = np.zeros((b, m, n)) if C is None else np.array(C, dtype=np.float64, order="C", copy=True)
    cin = None if Cin is None else np.ascontiguousarray(Cin, dtype=np.float64)
    st = _lib.sgs_kernel_gemm(_ptr(A), _ptr(B), _ptr(cin) if cin is not None else None, m, n, k, int(trans_a),
                              int(trans_b), alpha, beta, diag, mode + (4 if b_antisym else 0), gj[0], gj[1], b,
                              int(fp64_path), int(emulation_scratch), _ptr(out))
    if st != 0:
        raise SGSError(st, "batched gemm")
    return out
