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


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_roofline_flop_counts_per_evaluation():
    # sum-factorised contraction over (phi, theta, s): 2 (P + P_s P_ang + P_s) real FMAs
    # per right-hand side, plus the complex multiply-accumulate by the factor; the adjoint's
    # rank-1 update: P real-by-complex multiply-adds plus one complex product
    b = _bench_module()
    assert b.upward_flops_per_eval(3, 5) == 2 * 2 * (75 + 15 + 3) + 8 == 380
    assert b.upward_flops_per_eval(4, 7) == 2 * 2 * (196 + 28 + 4) + 8 == 920
    assert b.adjoint_flops_per_eval(3, 5) == 4 * 75 + 8 == 308
    assert b.adjoint_flops_per_eval(4, 7) == 4 * 196 + 8 == 792


def test_recorded_traffic_is_dropped_when_the_kernels_change(tmp_path):
    # a recorded DRAM figure is reported only for the kernel source it was measured on
    b = _bench_module()
    src = tmp_path / "kernels.cuh"
    src.write_text("// kernels\n")
    b.KERNEL_SOURCE = str(src)
    b.TRAFFIC_BYTES_PER_LAUNCH = {("w", "mixed"): {"bytes": 5.0e9, "sha": b._source_sha(str(src))}}
    assert b.traffic_per_launch("w", "mixed") == 5.0e9
    assert b.traffic_per_launch("w", "fp64") is None
    src.write_text("// kernels, changed\n")
    assert b.traffic_per_launch("w", "mixed") is None
