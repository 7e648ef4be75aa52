"""bench.py's reference arm on CPU: the FP64 oracle timed through
`bench.py --impl reference`, one JSON line with the benchmark line's keys;
under torch.distributed.run with two ranks, rank 0 alone runs and prints it.
Also the arithmetic of the per-stage rooflines."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def check_line(d, n_gpus):
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["n_gpus"] == n_gpus and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "sweeps/s" and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    check_line(lines[0], 1)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_two_ranks():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = json_lines(r.stdout)
    assert len(lines) == 1
    check_line(lines[0], 2)


def test_stage_rooflines_arithmetic():
    """The per-stage roofline figures from stage times, against hand arithmetic."""
    sys.path.insert(0, ROOT)
    import bench

    class W:
        n = m = 1 << 20

    prof = {"gather": (400, 100.0), "spread": (400, 90.0), "fft": (1200, 22.0),
            "direct": (2, 540.0), "bin": (4, 1.0)}
    peaks = {"hbm_gbs": 6774.0, "sm_max_mhz": 2070.0}
    plan = {"cutoff": 6, "grid": 128}
    r = bench.stage_rooflines(prof, W, 152, peaks, plan, (32.0, 123.0))
    clk = 2070e6
    t = 100.0e-3 / 400                                   # s per gather launch
    g = r["gather"]
    assert g["us_per_launch"] == pytest.approx(t * 1e6)
    assert g["achieved"] == pytest.approx((1 << 20) * 1728 / t / 1e9)
    assert g["peak"] == pytest.approx(123.0 * 152 * clk / 1e9)
    assert g["frac"] == pytest.approx(g["achieved"] / g["peak"])
    assert g["hbm"]["algorithmic_bytes"] == 16 * (1 << 20) + 4 * 128 ** 3
    assert g["share"] == pytest.approx(100.0 / 753.0)
    f = r["fft"]
    tf = 22.0e-3 / 1200
    assert f["bound"] == "hbm" and f["achieved"] == pytest.approx(2 * 4 * 128 ** 3 / tf / 1e9)
    d = r["direct"]
    assert d["achieved"] == pytest.approx((1 << 40) / (540.0e-3 / 2) / 1e9)
    assert d["peak"] == pytest.approx(32.0 * 152 * clk / 1e9)
    assert r["bin"]["achieved"] is None and "frac" not in r["bin"]
