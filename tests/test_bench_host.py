"""Host logic of bench.py (CPU): the reference arm's oracle sample calls the
oracle's own pair and state functions and scales them to the step, the
reference line carries the keys of the bench contract, and the roofline's
DRAM traffic is taken from a capture only while it describes the timed step."""
import json
import os
import subprocess
import sys

import numpy as np

import bench
from oracle import sgs_oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def perf_counter(self):
        return self.t


def test_oracle_sample_scales_pairs_and_states(monkeypatch):
    """A fake clock advanced by each oracle call: 1 per pair_elements, 0.5 per eom_term, 0.25 per
    orthogonal step and per purification.  A pair then costs 2 (its elements and both receivers'
    terms) and a state 1 (its own term and the update), and the step is 2 P + M."""
    clock = FakeClock()
    monkeypatch.setattr(bench, "time", clock)
    calls = []

    def pair_elements(model, gam, a, b):
        assert a < b
        calls.append(("pair", a, b))
        clock.t += 1.0
        return 1.0 + 0.0j, 0.0j

    def eom_term(model, gam, G, h, E, lam, mu, beta):
        calls.append(("eom", mu, beta))
        clock.t += 0.5
        return np.zeros_like(gam[0], dtype=np.complex128)

    def orthogonal_step(Gm, dG, ds):
        # the update direction is antisymmetric, as a step's dGamma is
        assert np.abs(dG + dG.T).max() == 0.0
        clock.t += 0.25
        return Gm

    def purify(Gm):
        clock.t += 0.25
        return Gm

    monkeypatch.setattr(orc, "pair_elements", pair_elements)
    monkeypatch.setattr(orc, "eom_term", eom_term)
    monkeypatch.setattr(orc, "orthogonal_step", orthogonal_step)
    monkeypatch.setattr(orc, "purify", purify)
    w = bench.workload("small")
    M = w.rank
    t_step, sample = bench.oracle_sample(w, n_pairs=3, n_states=2)
    assert t_step == 2.0 * M * (M - 1) / 2 + 1.0 * M
    assert f"{M * (M - 1) // 2} pairs + {M} states" in sample
    # every pair is followed by the terms of both its receivers; every state takes its own term
    pairs = [i for i, c in enumerate(calls) if c[0] == "pair"]
    assert len(pairs) == 3
    for i in pairs:
        _, a, b = calls[i]
        assert {calls[i + 1][1:], calls[i + 2][1:]} == {(b, a), (a, b)}
    own = [c for c in calls[pairs[-1] + 3:]]
    assert own == [("eom", 0, 0), ("eom", 1, 1)]


def test_reference_line_keys():
    """`bench.py --impl reference` prints one JSON line with the contract's keys; its value is the
    oracle's rate, echoed in cpu_baseline and e2e (no host-device copies)."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "steps/s"
    assert abs(d["ms_per_step"] * d["value"] - 1e3) < 1e-6 * 1e3
    assert d["config"]["workload"].startswith("anderson_L16_M4")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the oracle and prints; the other ranks exit 0 without work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "1",
                        "--warmup", "0", "--gpus", "2"], cwd=ROOT, capture_output=True, text=True, env=env,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def _traffic_file(tmp_path, sources_sha):
    src = tmp_path / "k.cu"
    src.write_text("kernel source")
    rec = {"oz_all_fp64": {"n": 512, "rank": 32, "panel_widths_gj_pf": [16, 16], "fp64_path": "emulated",
                           "launches_per_step": 92, "bytes_per_launch": 123.0,
                           "sources": {"k.cu": sources_sha(src)}}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    return str(f), src


def test_traffic_reported_only_for_the_captured_step(tmp_path):
    """The bench's `traffic` comes from the capture only for the captured shape, panel widths, FP64
    path and launch count, and only while the counted kernels' sources are unchanged."""
    f, src = _traffic_file(tmp_path, lambda p: bench._sha256(str(p)))
    root = str(tmp_path)
    base = dict(precision="fp64", fp64_path="emulated", n=512, rank=32, widths=[16, 16], launches=92 * 5, steps=5)
    assert bench.traffic_per_launch(f, root=root, **base) == 123.0
    for k, v in (("n", 256), ("rank", 12), ("widths", [12, 16]), ("fp64_path", "fma"), ("launches", 92 * 5 + 1),
                 ("precision", "tf32")):
        assert bench.traffic_per_launch(f, root=root, **dict(base, **{k: v})) is None, k
    src.write_text("kernel source, changed")
    assert bench.traffic_per_launch(f, root=root, **base) is None
    assert bench.traffic_per_launch(str(tmp_path / "absent.json"), root=root, **base) is None
