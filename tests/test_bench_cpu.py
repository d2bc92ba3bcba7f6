"""The benchmark's reference arm runs on the host cores alone (the FP64 oracle on a bounded pixel
sample of the paper-scale frame) and prints one JSON line with the keys the harness reads; the
error study's summary of GPU values against the oracle."""
import dataclasses
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "Mpixel/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("paper-scale")


def test_error_summary_of_the_oracle_against_itself_and_a_perturbed_copy():
    """The error study's summary: zero error for the oracle's own values, the planted relative
    error for a scaled copy, and mixed level counts (orders 0 and 2) summarised together."""
    import numpy as np
    import oracle
    from paper_1308_4908_gb300 import synth
    import bench
    parts = []
    for order in (0, 2):
        fr = synth.paper_scale(size=24, seed=3)
        p = dataclasses.replace(fr.params, order=order)
        pix = np.array([[u, v] for u in range(2, 22, 4) for v in range(3, 22, 5)])
        o = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
        gc = np.where(o["choice"] < 0, 255, o["choice"])
        parts.append((o["out"], gc, o))
    s = bench.error_stats(parts)
    assert s["n"] > 0 and s["max"] == 0.0 and s["level_mismatch_frac"] == 0.0 and s["nan_mismatch"] == 0
    scaled = [(g * (1 + 3e-6), gc, o) for g, gc, o in parts]
    s = bench.error_stats(scaled)
    big = np.concatenate([np.abs(o["out"]).ravel() for _, _, o in parts])
    big = big[np.isfinite(big)]
    want = (3e-6 * big / np.maximum(big, 1e-2)).max()
    assert s["max"] == pytest.approx(want, rel=1e-6) and s["frac_above_1e-5"] == 0.0
