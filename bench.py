#!/usr/bin/env python
"""Imaginary-time steps per second of the SGS variational method on GB300.

Workload: Anderson impurity, 127 bath sites per spin (N = 256 modes, 2N = 512),
rank M = 32, U = 4, eps_d = -2, V = 0.5, ds = 0.05, seeded random pure states.
A step is one pass of the whole hot path (pairs, amplitudes, equation of
motion, update, re-purification) over all M states.  Inputs stay resident in
HBM during the timed region (the per-step working set, several GB, is far
larger than L2).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|tf32]
  python bench.py --impl reference ...   (the FP64 CPU oracle on the host cores)

Prints one JSON line (rank 0).  The line's value is the FP64 step (every
product in FP64 arithmetic, emulated on the tensor cores: the library's
default); its "mixed" object times the TF32 form of the same workload in the
same run and states its energy and spin-correlator deviation from the FP64 run
over the same steps.  Under torchrun each rank runs its own replica of the
workload (independent problems, no collective on the data path).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sgs_inputs as inp  # noqa: E402

UNIT = "steps/s"
PRECISIONS = {"fp64": 0, "tf32": 1, "bf16": 2, "3xtf32": 3}
DTYPES = {"fp64": "f64", "tf32": "f64+tf32", "bf16": "f64+bf16", "3xtf32": "f64+3xtf32"}


def _sha256(path):
    import hashlib
    try:
        with open(path, "rb") as f:
            return hashlib.sha256(f.read()).hexdigest()
    except OSError:
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sgs", choices=["sgs", "reference"])
    ap.add_argument("--precision", default="fp64", choices=list(PRECISIONS))
    ap.add_argument("--workload", default="large",
                    choices=["large", "small", "two_channel", "siam_L500", "serving", "batched", "siam_estar"])
    ap.add_argument("--instances", type=int, default=256, help="batched: number of independent instances")
    ap.add_argument("--max-bath", type=int, default=64, help="batched: bath length L ~ U{16..max-bath}")
    ap.add_argument("--rate", type=float, default=100.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--requests", type=int, default=16, help="serving: number of requests")
    ap.add_argument("--max-steps", type=int, default=400, help="serving: step cap per solve")
    ap.add_argument("--serving-dtau", type=float, default=0.2, help="serving: imaginary-time step")
    ap.add_argument("--serving-mix", default="scaled", choices=["scaled", "configured"],
                    help="serving: request sizes L ~ U{8..40}, M in {4, 8} (scaled) or L ~ U{16..256}, "
                         "M in {8, 16, 32} (the batched workload's mix)")
    ap.add_argument("--rank", type=int, default=0, help="override the ansatz rank M (profiling cases)")
    ap.add_argument("--estar-rank", type=int, default=8, help="siam_estar: largest rank of the growth")
    ap.add_argument("--estar-steps", type=int, default=200, help="siam_estar: steps per rank")
    ap.add_argument("--estar-ds", type=float, default=0.1, help="siam_estar: imaginary-time step")
    ap.add_argument("--estar-knorm", type=float, default=0.1, help="siam_estar: ||K||_F of an added state's generator")
    ap.add_argument("--fp64-path", default="emulated", choices=["fma", "emulated"],
                    help="FP64 products: emulated on the bf16 tensor cores (the library's default) or FMA pipe")
    ap.add_argument("--emulation-scratch-gb", type=float, default=0.0,
                    help="emulated FP64 products: slice scratch per instance (GB; default 6 for one instance, "
                         "0.125 per instance for the batched and serving workloads)")
    ap.add_argument("--mixed", default="tf32", choices=["tf32", "bf16", "3xtf32", "none"],
                    help="mixed-precision form timed beside the FP64 line (the line's 'mixed' object)")
    ap.add_argument("--panel-widths", default="",
                    help="GJ,PF: fix the factorisation panel widths after the autotuner (reproducible profiles)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--accuracy-steps", type=int, default=0,
                    help="run the FP64 form and --precision side by side for this many steps and report the "
                         "energy and spin-correlator differences (one JSON line)")
    return ap.parse_args()


def workload(name, rank=0):
    import dataclasses
    w = {"large": inp.LARGE, "small": inp.SMALL, "two_channel": inp.TWO_CHANNEL, "siam_L500": inp.SIAM_L500}[name]
    if rank > 0:
        w = dataclasses.replace(w, rank=rank, name=f"{w.name.rsplit('_M', 1)[0]}_M{rank}")
    return w


def config_of(w, precision):
    p = w.model
    chans = f"{p.n_channels} channels x " if p.n_channels > 1 else ""
    return {"workload": f"{w.name}: Anderson impurity, {chans}{p.n_bath} bath sites/spin, 2N={2 * p.n_modes}, "
                        f"M={w.rank}, U={p.U}, eps_d={p.eps_d}, V={p.V}, t={p.t}, ds={w.dtau}",
            "n": 2 * p.n_modes, "rank": w.rank, "precision": precision, "seed": w.seed,
            "l2": "inputs larger than L2 (per-step working set of several GB, no flush needed)",
            "inputs": "seeded random pure states Gamma = O J O^T, O Haar on O(2N)"}


# --------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- CPU oracle sample

def oracle_sample(w, n_pairs=4, n_states=1):
    """Time the FP64 oracle, as it stands, on a bounded sample of one step of
    the workload: n_pairs pair evaluations (the oracle's pair_elements: overlap
    with phase, transition matrix, Wick energy; and its eom_term for both
    receivers of the pair) and n_states state evaluations (eom_term of the
    state's own term, orthogonal step, purification), then scale to the step's
    M(M-1)/2 pairs and M states.  Returns (seconds per step, sample)."""
    from oracle import sgs_oracle as orc
    p = w.model
    model = orc.anderson_model(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels)
    m = max(n_pairs + 1, n_states + 1, 2)
    g, _ = inp.initial_state(p.n_modes, m, w.seed, w.parity)
    gam = list(g)
    # the amplitude problem's values only scale the terms: unit Gram matrix and amplitudes
    G = np.eye(m, dtype=np.complex128)
    h = np.zeros((m, m), dtype=np.complex128)
    lam = np.ones(m, dtype=np.complex128)
    t0 = time.perf_counter()
    for k in range(n_pairs):
        a, b = 1 + (k % (m - 1)), 1 + ((k + 1) % (m - 1))
        if a == b:
            b = 0
        a, b = min(a, b), max(a, b)
        G[a, b], h[b, a] = orc.pair_elements(model, gam, a, b)
        orc.eom_term(model, gam, G, h, 0.0, lam, b, a)      # both receivers of the pair
        orc.eom_term(model, gam, G, h, 0.0, lam, a, b)
    t_pairs = (time.perf_counter() - t0) / n_pairs
    t0 = time.perf_counter()
    for k in range(n_states):
        orc.eom_term(model, gam, G, h, 0.0, lam, k, k)
        # a tangent direction of the same size as a step's: the commutator of two states
        dG = 0.01 * (gam[k] @ gam[k + 1] - gam[k + 1] @ gam[k])
        orc.purify(orc.orthogonal_step(gam[k], dG, w.dtau))
    t_states = (time.perf_counter() - t0) / n_states
    M = w.rank
    t_step = t_pairs * M * (M - 1) / 2 + t_states * M
    sample = (f"{n_pairs} pair evaluations + {n_states} state evaluation(s) of the {w.name} step, "
              f"scaled to {M * (M - 1) // 2} pairs + {M} states")
    return t_step, sample


def cpu_cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count()


# --------------------------------------------------------------------- arms

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload(args.workload, args.rank)
    for _ in range(args.warmup):
        oracle_sample(w, n_pairs=1, n_states=1)
    times = []
    sample = ""
    for _ in range(args.steps):
        t, sample = oracle_sample(w, n_pairs=4, n_states=1)
        times.append(t)
    t_step = float(np.mean(times))
    value = 1.0 / t_step
    line = {"impl": "reference", "metric": f"imag-time steps/s at 2N={2 * w.model.n_modes},M={w.rank}", "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, "fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": "per timed step: " + sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


FP64_PATHS = {"emulated": 0, "fma": 1}


def traffic_per_launch(tfile, precision, fp64_path, n, rank, widths, launches, steps, root=ROOT):
    """DRAM bytes per FP64 product call from a committed ncu capture, or None.
    The counters hold for the same shape, panel widths and FP64 path only, for
    the same launch sequence (a changed step shows as another launch count),
    and only while the sources of the counted kernels are the ones captured."""
    if not os.path.exists(tfile):
        return None
    try:
        with open(tfile) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    key = f"oz_all_{precision}" if fp64_path == "emulated" else f"gemm_f64_all_{precision}"
    t = rec.get(key)
    if not t or not t.get("sources"):
        return None
    fresh = all(_sha256(os.path.join(root, f)) == hsh for f, hsh in t["sources"].items())
    if (fresh and t.get("n") == n and t.get("rank") == rank and t.get("fp64_path") == fp64_path
            and t.get("panel_widths_gj_pf") == list(widths)
            and t.get("launches_per_step", -1) * steps == launches):
        return t.get("bytes_per_launch")
    return None


def path_kwargs(args):
    """Solver options for the FP64 products: the path and, when emulated, the slice scratch."""
    gb = args.emulation_scratch_gb or (0.125 if args.workload in ("batched", "serving") else 6.0)
    return {"fp64_path": FP64_PATHS[args.fp64_path],
            "emulation_scratch": int(gb * 1e9) if args.fp64_path == "emulated" else 0}


def dtype_of(args, precision=None):
    d = DTYPES[precision or args.precision]
    return d.replace("f64", "f64e", 1) if args.fp64_path == "emulated" else d


def tc_roofline(prof, precision, n, pairs, steps, peaks):
    """Roofline of the tensor-core V = D W product of the mixed forms (per pair 2 n^3
    flops; algorithmic bytes = the two operands read once, hi and lo parts for 3xTF32,
    and the fp32 product written once), from one profiled region of `steps` steps."""
    if precision == "fp64" or prof["eom_v"][0] <= 0:
        return None
    bf16 = peaks.get("bf16_tflops", 1900.0)
    hbm = peaks.get("hbm_gbs", 6800.0)
    ratio = {"tf32": 1.1 / 2.25, "3xtf32": 1.1 / 2.25 / 3.0, "bf16": 1.0}[precision]
    tc_peak = bf16 * ratio
    v_ms, v_fl, _ = prof["eom_v"]
    ldp = (n + 7) // 8 * 8
    esz = 2 if precision == "bf16" else 4
    parts = 2 if precision == "3xtf32" else 1
    v_bytes = pairs * (2.0 * parts * n * ldp * esz + 4.0 * n * n) * steps
    flops_s = v_fl / (v_ms * 1e-3)
    bytes_s = v_bytes / (v_ms * 1e-3)
    intensity = v_fl / v_bytes
    hbm_bound = intensity * hbm * 1e9 / 1e12 < tc_peak
    return {"bound": "hbm" if hbm_bound else "tensor",
            "kernel": f"gemm_tma_kernel (TMA-fed tcgen05 {precision}, V = D W)",
            "achieved": bytes_s / 1e9 if hbm_bound else flops_s / 1e12,
            "peak": hbm if hbm_bound else tc_peak, "unit": "GB/s" if hbm_bound else "TFLOP/s",
            "frac": (bytes_s / 1e9 / hbm) if hbm_bound else (flops_s / 1e12 / tc_peak),
            "tflops": flops_s / 1e12, "tensor_peak_tflops": tc_peak,
            "arithmetic_intensity_flops_per_byte": intensity,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs; tensor peak = bf16_tflops x nominal ratio "
                           f"({precision}: {ratio:.3f})"}


def timed_steps(torch, solver, stream, args, dist, local):
    """Warm-up steps, then exactly args.steps steps between barriers and synchronisations,
    CUDA events on the solver's stream and nvidia-smi clocks sampled meanwhile.  Returns
    (energies of every step run, warm-up included, ms of the timed steps, clocks, the library's
    kernel launches in the timed steps)."""
    Ew = solver.step(args.warmup)
    solver.set_profiling(False)                   # resets the launch counter (profiling stays off)
    clocks = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    E = solver.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    return np.concatenate([Ew[0], E[0]]), e0.elapsed_time(e1), ck, solver.profile()[1]


def run_sgs(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2105_01088_gb300 as sgs

    sgs.use_torch_allocator()
    w = workload(args.workload, args.rank)
    p = w.model
    prec = PRECISIONS[args.precision]
    g, lam = inp.initial_state(p.n_modes, w.rank, w.seed + 1000 * rank, w.parity)
    model = sgs.build_anderson(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels)
    stream = torch.cuda.Stream()          # a capturable stream: steps replay a CUDA graph
    solver = sgs.Solver(model, g, lam, dtau=w.dtau, precision=prec, parity=w.parity, stream=stream, autotune=True,
                        **path_kwargs(args))
    if args.panel_widths:
        solver.set_panel_widths(*[int(x) for x in args.panel_widths.split(",")])
    metric = f"imag-time steps/s at 2N={2 * p.n_modes},M={w.rank}"
    peak_fp64_fma = sgs.probe_peak(1)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    # the emulated path issues 36 bf16 slice products per FP64 product: its ceiling is the
    # measured bf16 rate / 36
    peak_fp64 = {"fma": peak_fp64_fma, "emulated": peaks.get("bf16_tflops", 1900.0) / 36.0}[args.fp64_path]

    E_all, ms, ck, launches_timed = timed_steps(torch, solver, stream, args, dist, local)
    sites = list(range(0, min(p.n_bath + 1, 33)))
    C_main = solver.correlator(sgs.SGS_CORR_SPIN_SPIN, sites)
    # second timed region of the same length with per-stage and per-GEMM-launch events (direct
    # launches) for the roofline of the dominant kernel
    solver.set_profiling(True)
    solver.step(args.steps)
    prof, _, gemm_prof = solver.profile()
    solver.set_profiling(False)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * args.steps / (ms_max * 1e-3)

    # end to end through the public API with pinned host buffers
    n = 2 * p.n_modes
    g_host = torch.empty((w.rank, n, n), dtype=torch.float64, pin_memory=True).numpy()
    g_host[:] = solver.get_state()[0]
    lam_host = np.zeros(w.rank, complex)
    k_e2e = max(1, min(args.steps, 3))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        solver.set_state(g_host, None)
        solver.step(1)
        _, lam_host[:] = solver.get_state(out=g_host)
    t_e2e = time.perf_counter() - t0
    te = torch.tensor([t_e2e], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = world * k_e2e / float(te.item())
    h2d = w.rank * n * n * 8
    d2h = w.rank * n * n * 8 + w.rank * 16 + 8

    # roofline of the dominant kernel: every FP64 product of the step (all launches), algorithmic
    # flops of all its launches / their summed time
    g_ms, g_fl, g_n = gemm_prof
    roof = None
    if g_ms > 0:
        achieved = g_fl / (g_ms * 1e-3) / 1e12
        traffic = traffic_per_launch(os.path.join(ROOT, "profiles", "traffic.json"), args.precision,
                                     args.fp64_path, n, w.rank, list(solver.tuning(0)[:2]), int(g_n), args.steps)
        if args.fp64_path == "emulated":
            kern = ("oz_gemm_kernel with its slicing kernels (FP64 products emulated on the bf16 tensor cores; "
                    "all FP64 products: Gauss-Jordan and Pfaffian updates, pair and state products)")
            src = ("MEASURED_PEAKS.json bf16_tflops / 36 (36 bf16 slice products per FP64 product); achieved = "
                   "algorithmic FP64 flops / time of the products including slicing")
        else:
            kern = ("gemm_f64_kernel (FP64 FMA; all its launches: Gauss-Jordan and Pfaffian updates, pair and "
                    "state products)")
            src = "measured live: FP64 FMA throughput probe (sgs_probe_peak kind 1); not in MEASURED_PEAKS.json"
        roof = {"bound": "alu" if args.fp64_path == "fma" else "tensor", "achieved": achieved, "peak": peak_fp64,
                "unit": "TFLOP/s", "frac": achieved / peak_fp64, "traffic": traffic, "kernel": kern,
                "launches": int(g_n), "flops_per_launch": g_fl / max(g_n, 1), "ms_per_launch": g_ms / max(g_n, 1),
                "peak_source": src}
    pairs = w.rank * (w.rank - 1) // 2
    stages = {s: {"ms_per_step": v[0] / args.steps, "tflops": (v[1] / (v[0] * 1e-3) / 1e12) if v[0] > 0 and v[1] > 0
                  else None} for s, v in prof.items()}
    line = {"metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_of(args), "data": "synthetic",
            "config": dict(config_of(w, args.precision), fp64_products=args.fp64_path),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches_timed), "roofline": roof,
            "tc_roofline": tc_roofline(prof, args.precision, n, pairs, args.steps, peaks), "clocks": ck,
            "stages": stages, "energy_last": float(E_all[-1]), "panel_widths_gj_pf": list(solver.tuning(0)[:2]),
            "fp64_fma_peak_tflops": peak_fp64_fma}
    solver.close()

    # the mixed form of the same workload from the same states: the same warm-up and timed steps
    if args.mixed != "none" and args.precision == "fp64":
        ms_solver = sgs.Solver(model, g, lam, dtau=w.dtau, precision=PRECISIONS[args.mixed], parity=w.parity,
                               stream=stream, autotune=True, **path_kwargs(args))
        if args.panel_widths:
            ms_solver.set_panel_widths(*[int(x) for x in args.panel_widths.split(",")])
        Em_all, ms_m, ck_m, _ = timed_steps(torch, ms_solver, stream, args, dist, local)
        C_mixed = ms_solver.correlator(sgs.SGS_CORR_SPIN_SPIN, sites)
        ms_solver.set_profiling(True)
        ms_solver.step(args.steps)
        prof_m, _, _ = ms_solver.profile()
        ms_solver.set_profiling(False)
        tm = torch.tensor([ms_m], dtype=torch.float64, device="cuda")
        if dist:
            dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        msm_max = float(tm.item())
        line["mixed"] = {
            "precision": args.mixed, "dtype": dtype_of(args, args.mixed),
            "value": world * args.steps / (msm_max * 1e-3), "unit": UNIT, "ms_per_step": msm_max / args.steps,
            "speedup_vs_fp64": ms_max / msm_max,
            "tc_roofline": tc_roofline(prof_m, args.mixed, n, pairs, args.steps, peaks), "clocks": ck_m,
            "stages": {s: {"ms_per_step": v[0] / args.steps} for s, v in prof_m.items()},
            "panel_widths_gj_pf": list(ms_solver.tuning(0)[:2]),
            "accuracy_vs_fp64": {
                "steps_compared": int(len(E_all)),
                "energy_rel_diff_max": float(np.max(np.abs(Em_all - E_all)) / np.max(np.abs(E_all))),
                "energy_rel_diff_last": float(abs(Em_all[-1] - E_all[-1]) / abs(E_all[-1])),
                "corr_sites": sites, "corr_abs_diff_max": float(np.max(np.abs(C_mixed - C_main))),
                "corr_max_abs": float(np.max(np.abs(C_main))),
                "note": "the same initial states, warm-up and timed steps on both forms; C(r) of the states "
                        "after the timed steps"}}
        ms_solver.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t_step, sample = oracle_sample(w, n_pairs=24, n_states=4)
        line["cpu_baseline"] = {"value": 1.0 / t_step, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                "sample": sample}
        # the same sample with one BLAS thread, in a child process (thread counts are fixed at import)
        env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
        code = ("import bench, sgs_inputs; w = bench.workload(%r, %d); "
                "t, s = bench.oracle_sample(w, n_pairs=8, n_states=2); print(t)" % (args.workload, args.rank))
        try:
            r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                               timeout=600)
            t1 = float(r.stdout.strip().splitlines()[-1])
            line["cpu_baseline_1_thread"] = {"value": 1.0 / t1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                             "sample": "8 pair evaluations + 2 state evaluations, scaled to the step"}
        except (subprocess.SubprocessError, ValueError, IndexError):
            line["cpu_baseline_1_thread"] = None
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def run_serving(args):
    """Continuous batching of a Poisson stream of impurity solves (mixed precision,
    resident slots admitted by an HBM budget) against the same solves run one at
    a time with the plain FP64 step."""
    import torch
    import paper_2105_01088_gb300 as sgs
    from paper_2105_01088_gb300.serving import Request, ServingLoop, latency_stats, run_sequential

    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    sgs.use_torch_allocator()
    prec = PRECISIONS[args.precision]
    reqs = []
    mix = dict(n_bath=(16, 256), ranks=(8, 16, 32)) if args.serving_mix == "configured" else {}
    for i, (t, p, M, seed, par) in enumerate(inp.serving_requests(args.rate, args.requests, seed=7, **mix)):
        if args.serving_mix == "configured":
            g, lam = clustered_states_device(p.n_modes, M, seed, par)
        else:
            g, lam = inp.initial_state(p.n_modes, M, seed, par)
        reqs.append(Request(i, t, sgs.build_anderson(p.n_bath, p.U, p.eps_d, p.V), g, lam, par))
    stream = torch.cuda.Stream()
    budget = int(torch.cuda.get_device_properties(0).total_memory * 0.5)
    # warm-up: one solve in each mode (kernel loading, allocator pools)
    for pr in (prec, 0):
        w = sgs.Solver(stream=stream, **path_kwargs(args))
        k = w.admit(reqs[0].model, reqs[0].gamma0, reqs[0].lambda0, 0.05, pr, 0, reqs[0].parity)
        w.step(3)
        w.close()
    solver = sgs.Solver(stream=stream, hbm_budget=budget, **path_kwargs(args))
    # phase form of c_mu (Sec. III A): with the inverse form, random initial states (amplitudes down to
    # 1e-14) drive steps outside the exponential's range at these step sizes
    loop = ServingLoop(solver, dtau=args.serving_dtau, precision=prec, cmode=1, tol=1e-8, max_steps=args.max_steps)
    res = loop.run(reqs)
    solver.close()
    seq = run_sequential(lambda: sgs.Solver(stream=stream, **path_kwargs(args)), reqs, dtau=args.serving_dtau, precision=0, cmode=1,
                         tol=1e-8, max_steps=args.max_steps)
    a, b = latency_stats(res), latency_stats(seq)
    dE = max((abs(x.energy - y.energy) / abs(y.energy) for x, y in zip(res, seq)
              if np.isfinite(x.energy) and np.isfinite(y.energy)), default=float("nan"))
    line = {"metric": "impurity solves/s (continuous batching, Poisson arrivals)", "value": a["throughput_per_s"],
            "unit": "solves/s", "n_gpus": 1, "steps": int(sum(r.steps for r in res)), "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(args), "data": "synthetic",
            "config": {"workload": f"serving: {args.requests} Anderson solves, Poisson rate {args.rate}/s, "
                                   + ("bath L ~ U{16..256}, M in {8, 16, 32} (clustered initial states)"
                                      if args.serving_mix == "configured" else "bath L ~ U{8..40}, M in {4, 8}")
                                   + ", U ~ U[0,8], V ~ U[0.2,1], run to |dE| < 1e-8 "
                                   f"per step or {args.max_steps} steps at ds = {args.serving_dtau}, phase form of c_mu",
                       "hbm_budget_bytes": budget},
            "latency": {"p50_s": a["p50_s"], "p99_s": a["p99_s"], "mean_s": a["mean_s"]},
            "sequential_fp64": {"throughput_per_s": b["throughput_per_s"], "p50_s": b["p50_s"], "p99_s": b["p99_s"]},
            "converged": int(sum(r.converged for r in res)), "failed": len(loop.failures),
            "max_rel_energy_diff_vs_sequential_fp64": dE}
    print(json.dumps(line))
    return 0


def clustered_states_device(n_modes, M, seed, parity, spread=1.0):
    """The clustered pure states of sgs_inputs.clustered_pure_gammas (Gamma_mu = O_mu Gamma_0 O_mu^T,
    O_mu = exp(K_mu), K_mu antisymmetric N(0, (spread / n)^2), Gamma_0 = O J O^T with O Haar from
    the QR of a normal matrix, the first column negated for the parity), drawn with a seeded torch
    generator on the device: the host's dense exponentials of n ~ 1000 matrices would take longer
    than the benchmark.  Returns host arrays (gamma [M, n, n], lambda [M])."""
    import torch
    n = 2 * n_modes
    gen = torch.Generator(device="cuda").manual_seed(int(seed))
    X = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=gen)
    Q, R = torch.linalg.qr(X)
    Q = Q * torch.sign(torch.diagonal(R))
    if (torch.linalg.det(Q) > 0) != (parity > 0):
        Q[:, 0] = -Q[:, 0]
    J = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    idx = torch.arange(0, n, 2, device="cuda")
    J[idx, idx + 1] = 1.0
    J[idx + 1, idx] = -1.0
    base = Q @ J @ Q.T
    out = []
    for _ in range(M):
        K = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=gen) * (spread / n)
        O = torch.linalg.matrix_exp(K - K.T)
        G = O @ base @ O.T
        out.append(0.5 * (G - G.T))
    g = torch.stack(out).cpu().numpy()
    th = torch.rand(M, dtype=torch.float64, device="cuda", generator=gen).cpu().numpy() * 2.0 * np.pi
    return np.ascontiguousarray(g), np.exp(1j * th)


def run_estar(args):
    """The ground-state energy estimate of Sec. IV A on its system (SIAM, L = 500 sites, U = t = 1,
    U / Gamma = 5, particle-hole symmetric), bounded: the rank grows from 1 to --estar-rank by the
    schedule of Sec. III C (growth.grow), --estar-steps steps per rank from the U = 0 ground state
    (one Gaussian, +-polar(A): the sign of lower energy), the variance delta_H^2 (Eq. residual) at
    the end of each rank, and E* the intercept of the linear fit of E against delta_H^2 over the
    ranks (growth.extrapolate_energy; the paper fits only points below 2e-5)."""
    import torch
    import paper_2105_01088_gb300 as sgs
    from paper_2105_01088_gb300.growth import extrapolate_energy, grow

    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    sgs.use_torch_allocator()
    p = inp.SIAM_L500.model
    model = sgs.build_anderson(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels)
    # the U = 0 ground state: Gamma = +-A |A|^-1 (the polar factor of A), the sign of the lower energy
    A = torch.tensor(model.A, dtype=torch.float64, device="cuda")
    U_, _, Vh = torch.linalg.svd(A)
    P = (U_ @ Vh).cpu().numpy()
    P = 0.5 * (P - P.T)
    stream = torch.cuda.Stream()
    best = None
    for sign in (1.0, -1.0):
        g = (sign * P)[None]
        ph, _ = sgs.batched_pfaffian(g.astype(np.complex128))
        parity = 1 if ph[0].real > 0 else -1
        s = sgs.Solver(model, g, None, dtau=args.estar_ds, parity=parity, stream=stream, cmode=1)
        e = s.variance(0)[0]                  # <H> of the current state, computed on the device
        s.close()
        if best is None or e < best[0]:
            best = (e, g, parity)
    e0, g0, parity = best
    solver = sgs.Solver(model, g0, None, dtau=args.estar_ds, parity=parity, stream=stream, cmode=1,
                        **path_kwargs(args))
    rng = np.random.default_rng(11)
    t0 = time.perf_counter()
    out = grow(solver, 0, args.estar_rank, args.estar_steps, args.estar_knorm, rng, with_variance=True)
    wall = time.perf_counter() - t0
    solver.close()
    ranks = [int(r) for r, _, _ in out]
    ev = [(float(v[0]), float(v[1])) for _, _, v in out]
    E = [x[0] for x in ev]
    var = [x[1] for x in ev]
    try:
        est, sigma = extrapolate_energy(E, var, var_max=float("inf"))
    except ValueError:
        est, sigma = float("nan"), float("nan")
    paper = -635.3490861
    line = {"metric": "ground-state energy estimate E* (Sec. IV A)", "value": est, "unit": "t",
            "sigma": sigma, "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
            "dtype": dtype_of(args),
            "config": {"workload": f"SIAM L = 500 (2N = 2000), U = t = 1, U/Gamma = 5, eps_d = -U/2, mu = 0; ranks 1.."
                                   f"{args.estar_rank}, {args.estar_steps} steps per rank at ds = {args.estar_ds}, "
                                   f"||K||_F = {args.estar_knorm}, phase form of c_mu, from the U = 0 ground state",
                       "fit": "all ranks (the paper fits only delta_H^2 < 2e-5)"},
            "paper_E_star": paper, "paper_sigma": 4e-7, "difference_to_paper": est - paper,
            "ranks": ranks, "energies": E, "variances": var, "E_U0_state": e0, "wall_s": wall,
            "steps": int(sum(len(x[1]) for x in out))}
    print(json.dumps(line))
    return 0


def run_batched(args):
    """Many independent uneven instances advanced together: every step replays one
    captured graph whose branches are the instances (their kernels overlap on the
    device).  Instances that do not fit the device together run in waves: each wave
    admits instances in order while they fit an HBM budget, takes the warm-up and the
    timed steps, and is released.  Instances are dealt round-robin to ranks (no
    collective)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2105_01088_gb300 as sgs

    sgs.use_torch_allocator()
    prec = PRECISIONS[args.precision]
    ws = inp.batched_workloads(args.instances, n_bath=(16, args.max_bath))
    mine = ws[rank::world]
    stream = torch.cuda.Stream()
    budget = int(torch.cuda.mem_get_info()[0] * 0.8)
    autotune = args.max_bath <= 64          # the capped default tunes each shape; the full range takes defaults
    ms_total, waves, launches, finite, shapes = 0.0, [], 0, True, {}
    flops_per_step = 0.0
    ck = None
    pending = list(mine)
    while pending:
        solver = sgs.Solver(stream=stream, autotune=autotune, hbm_budget=budget, **path_kwargs(args))
        wave = []
        while pending:
            w = pending[0]
            p = w.model
            # clustered states (order-one overlaps, as rank growth produces them): random pure states
            # of unrelated orientation give amplitudes near 1e-14, whose c_mu = 1/(lambda lambda-tilde*)
            # turns the first steps into rotations far outside a small step
            if args.max_bath <= 64:
                rng = np.random.default_rng(w.seed)
                g = inp.clustered_pure_gammas(p.n_modes, w.rank, rng, w.parity, spread=1.0)
                lam = inp.random_amplitudes(w.rank, rng)
            else:
                g, lam = clustered_states_device(p.n_modes, w.rank, w.seed, w.parity)
            # phase form of c_mu (Sec. III A): the inverse form divides by the amplitude, and from these
            # starts it drives rotations with ||X||_F of 1e2..1e3 per step
            try:
                solver.admit(sgs.build_anderson(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels), g, lam,
                             w.dtau, prec, 1, w.parity)
            except sgs.SGSError as e:
                if e.status == 2 and wave:
                    break                   # the budget is full: run this wave
                raise
            pending.pop(0)
            wave.append(w)
            n, M = 2 * p.n_modes, w.rank
            # dense work per step (the algorithmic count of the pair and state stages, in n^3 units)
            flops_per_step += n ** 3 * (M * (M - 1) / 2 * (2 + 1 + 4 / 3 + 1 + 2 + 1) * 2 + M * 60)
        solver.step(args.warmup)
        solver.set_profiling(False)           # resets the launch counter; graphs stay on
        clocks = ClockSampler(local)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        clocks.start()
        e0.record(stream)
        E = solver.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        wck = clocks.stop()
        ck = wck if ck is None or (wck.get("sm_mhz") or 0) < (ck.get("sm_mhz") or 1e9) else ck
        ms = e0.elapsed_time(e1)
        ms_total += ms
        launches += solver.profile()[1]
        finite = finite and bool(np.isfinite(E).all())
        for k in range(solver.n_instances):
            gj, pf, _ = solver.tuning(k)
            shapes[f"{gj}/{pf}"] = shapes.get(f"{gj}/{pf}", 0) + 1
        waves.append({"instances": len(wave), "bytes": solver.bytes_in_use(), "ms_per_step": ms / args.steps})
        solver.close()
    if dist:
        dist.barrier()
    t = torch.tensor([ms_total], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = len(ws) * args.steps / (ms_max * 1e-3)
    ns = [2 * w.model.n_modes for w in ws]
    line = {"metric": "instance-steps/s (batched uneven impurity instances)", "value": value,
            "unit": "instance-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": dtype_of(args), "data": "synthetic",
            "config": {"workload": f"batched: {len(ws)} Anderson instances, bath L ~ U{{16..{args.max_bath}}}, "
                                   "M in {8,16,32}, U ~ U[0,8], eps_d = -U/2, V ~ U[0.2,1], ds = 0.05",
                       "n_range": [min(ns), max(ns)], "precision": args.precision,
                       "inputs": "clustered pure states O_mu = exp(K_mu) O around one Haar O, random phases"
                                 + ("" if args.max_bath <= 64 else " (drawn on the device with a seeded torch generator)"),
                       "c_mu": "phase form (Sec. III A)", "autotune": autotune,
                       "hbm_budget_bytes": budget,
                       "waves": waves,
                       "timed": "the steps of each wave (CUDA events on the library's stream); admission excluded",
                       "l2": "inputs larger than L2 (tens of GB resident)"},
            "gpu_launches": launches, "clocks": ck, "all_energies_finite": finite,
            "panel_widths_gj_pf": shapes,
            "dense_tflops_per_s": flops_per_step / max(len(mine), 1) * len(ws) * args.steps / (ms_max * 1e-3) / 1e12}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


def run_accuracy(args):
    """The mixed form against the FP64 form over many steps from identical inputs: the
    final energy and the spin-spin correlator C(r) of the final states.  The FP64 form
    is checked against the oracle step by step by the parity tests."""
    import torch
    import paper_2105_01088_gb300 as sgs
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    sgs.use_torch_allocator()
    w = workload(args.workload, args.rank)
    p = w.model
    g, lam = inp.initial_state(p.n_modes, w.rank, w.seed, w.parity)
    model = sgs.build_anderson(p.n_bath, p.U, p.eps_d, p.V, p.t, p.mu, p.n_channels)
    stream = torch.cuda.Stream()
    sites = list(range(0, min(p.n_bath + 1, 33)))
    out = {}
    for name, prec in (("fp64", 0), (args.precision, PRECISIONS[args.precision])):
        s = sgs.Solver(model, g, lam, dtau=w.dtau, precision=prec, parity=w.parity, stream=stream, autotune=True)
        t0 = time.perf_counter()
        E = s.step(args.accuracy_steps)[0]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        C = s.correlator(sgs.SGS_CORR_SPIN_SPIN, sites)
        s.close()
        out[name] = (E, C, dt)
    E64, C64, _ = out["fp64"]
    Em, Cm, _ = out[args.precision]
    line = {"metric": "mixed vs FP64 accuracy over a trajectory", "workload": w.name, "steps": args.accuracy_steps,
            "precision": args.precision, "E_fp64_final": float(E64[-1]), f"E_{args.precision}_final": float(Em[-1]),
            "energy_rel_diff_final": float(abs(Em[-1] - E64[-1]) / abs(E64[-1])),
            "energy_rel_diff_max": float(np.max(np.abs(Em - E64)) / np.max(np.abs(E64))),
            "corr_sites": sites, "C_fp64": [float(x) for x in C64],
            "corr_abs_diff_max": float(np.max(np.abs(Cm - C64))),
            "seconds": {k: v[2] for k, v in out.items()}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.accuracy_steps > 0:
        return run_accuracy(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "siam_estar":
        return run_estar(args)
    return run_sgs(args)


if __name__ == "__main__":
    sys.exit(main())
