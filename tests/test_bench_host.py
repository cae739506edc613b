"""bench.py contract pieces that run without a GPU: the reference arm (the
FP64 oracle timed on the host cores) prints one JSON line with the agreed
keys, and ranks other than 0 print nothing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None):
    env = dict(os.environ)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        env.pop(k, None)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                           "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=300)


def test_reference_arm_json_line():
    r = _run()
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_are_silent():
    r = _run({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_roofline_kernel_name_and_traffic_record():
    """The roofline names the kernel the headline run launches, and the
    committed ncu traffic record applies only to that kernel on the current
    sources."""
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    def name(**kw):
        a = argparse.Namespace(**{"kernel": "auto", "dtype": "f32", "variant": "B", **kw})
        return bench.step_kernel_name(a)

    assert name() == "step_rows"
    assert name(dtype="f16") == "step_tma"
    assert name(dtype="f16", variant="lbgk") == "step_rows"
    assert name(kernel="rows", dtype="f16") == "step_rows"
    assert name(kernel="bulk") == "step_tma" and name(kernel="nodes") == "step_nodes"
    n = 16384
    t = bench.traffic_from_profile("step_rows<B,f32>", "f32", n)
    with open(os.path.join(ROOT, "profiles", "kbc_step_rows_f32_traffic.txt")) as f:
        current = f"kernel_source_hash: {bench.kernel_source_hash()}" in f.read()
    if current:
        assert t is not None and 70 * n * n < t <= 72 * n * n
    else:  # sources changed since the capture: no stale figure is reported
        assert t is None
    assert bench.traffic_from_profile("step_rows<C,f32>", "f32", n) is None
    assert bench.traffic_from_profile("step_tma<B,f32>", "f32", n) is None
    assert bench.traffic_from_profile("step_tma<B,f16>", "f16", n) is None


def test_fp64_ops_record_applies_to_its_kernel_only():
    """The FP64 path's roofline uses the committed FP64 instruction count only
    for the kernel it was captured on, on the current sources."""
    sys.path.insert(0, ROOT)
    import bench

    ops = bench.fp64_ops_from_profile("step_rows<B,f64>")
    with open(os.path.join(ROOT, "profiles", "kbc_step_rows_f64_ops.txt")) as f:
        current = f"kernel_source_hash: {bench.kernel_source_hash()}" in f.read()
    if current:
        assert ops is not None and 150 < ops < 260
    else:
        assert ops is None
    assert bench.fp64_ops_from_profile("step_rows<C,f64>") is None
