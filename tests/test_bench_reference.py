"""bench.py's reference arm on CPU: the JSON line of the FP64 direct sum on sampled
targets and of the oracle's serial IFGF, with the keys the benchmark contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(*extra):
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "sphere_4lambda", "--steps", "1", "--warmup", "0", *extra],
                       env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_direct_sum_line():
    d = _run("--ref-targets", "8")
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "8 sampled targets" in d["cpu_baseline"]["sample"]


def test_reference_serial_ifgf_line():
    d = _run("--ref-kind", "ifgf")
    assert KEYS <= set(d)
    assert d["config"]["reference"] == "oracle IFGF" and d["t_pre_ms"] > 0
    assert d["cpu_baseline"]["cores"] == 2
    assert abs(d["value"] - 24576 ** 2 / (d["ms_per_step"] * 1e-3)) < 1e-6 * d["value"]
