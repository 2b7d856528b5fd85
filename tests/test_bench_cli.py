"""bench.py's host side without a GPU: the per-workload serving shape, the CPU-baseline worker
and the reference arm's JSON line (the oracle, timed on the host, on the small workload)."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _args(*argv):
    old = sys.argv
    sys.argv = ["bench.py", *argv]
    try:
        return bench._args()
    finally:
        sys.argv = old


def test_serving_shape_defaults_per_workload():
    a = _args()
    assert (a.workload, a.chains, a.depth) == ("cfg2-fp32", 4, 4)
    a = _args("--workload", "cfg1-fp32")
    assert (a.chains, a.depth) == bench.SERVING_SHAPE["cfg1-fp32"]
    a = _args("--workload", "cfg3-bf16")
    assert (a.chains, a.depth) == bench.SERVING_SHAPE["cfg3-bf16"] == (3, 6)
    a = _args("--workload", "cfg3-bf16", "--chains", "1", "--depth", "2")
    assert (a.chains, a.depth) == (1, 2)
    assert a.steps >= 1 and a.warmup >= 3


def test_cpu_worker_runs_whole_frames_until_the_budget():
    n, secs = bench._oracle_seconds("cfg1-fp32", 0.0)
    assert n == 1 and secs > 0          # at least one frame, even with no budget
    n, secs = bench._oracle_seconds("cfg1-fp32", 1e9, max_frames=2)
    assert n == 2 and secs > 0          # bounded by the frame cap


@pytest.mark.timeout(300)
def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "cfg1-fp32", "--steps", "1", "--warmup", "3"],
                         capture_output=True, text=True, cwd=ROOT, timeout=280,
                         env=dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1"))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "frames/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["metric"] == "pillar frames/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_sweep_points_parse_positional_and_keyed():
    p = bench.parse_sweep_item("33:96:8:mixed:1:tight=0.4")
    assert (p["chains"], p["rate"], p["seconds"], p["mixed"], p["dfac"], p["tight"]) == (33, 96.0, 8.0, True, 1.0, 0.4)
    p = bench.parse_sweep_item("33:64:3:mixed:0.005:0.1")
    assert (p["dfac"], p["noise"], p["tight"], p["synth"]) == (0.005, 0.1, 0.0, None)
    p = bench.parse_sweep_item("33:5:3:mixed:0.1:0:0.5/100/1000")
    assert p["synth"] == (0.5, 100.0, 1000.0)
    p = bench.parse_sweep_item("11:1:4:bf16:tight=1:dfac=0.5")
    assert not p["mixed"] and p["dfac"] == 0.5 and p["tight"] == 1.0
    for bad in ("33:96", "33:96:8:mixed:tight=1.5", "33:96:8:tightness=0.4"):
        with pytest.raises(ValueError):
            bench.parse_sweep_item(bad)


def test_default_serving_points_are_past_plain_saturation_with_tight_share():
    """The default run's overload points use the paper's default share of tight-deadline chains
    (40 %) and replay at least 8 s each."""
    pts = {k: v for k, *v in bench.SERVING_POINTS}
    assert pts["config4_11_chains_1x"] == [11, 1.0, 4.0, False, 1.0, 0.0]
    over = [v for k, v in pts.items() if k != "config4_11_chains_1x"]
    assert over and all(n == 33 and secs >= 8.0 and tight == 0.4 for n, rate, secs, mixed, dfac, tight in over)


def test_clock_samples_go_to_the_chosen_directory(tmp_path):
    """The timed region's nvidia-smi samples are written under --clocks-dir (default: the system
    temporary directory), never into the source tree; without nvidia-smi the line says so."""
    a = _args("--clocks-dir", str(tmp_path))
    assert a.clocks_dir == str(tmp_path)
    assert _args().clocks_dir is None
    c = bench._Clocks(0, enabled=True, max_s=5.0, out_dir=str(tmp_path))
    try:
        assert os.path.dirname(c.path) == str(tmp_path) and os.path.exists(c.path)
    finally:
        r = c.stop()
    assert set(r) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    d = bench._Clocks(0, enabled=False)
    assert not os.path.commonpath([d.path, ROOT]) == ROOT
    d.stop()
