"""bench.py's contract on a machine without a GPU: the reference arm (the oracle on the
host cores) prints one JSON line with the contract's keys, and the GPU arm refuses to run
rather than fall back to the CPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_the_contract_line():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0", "--npts", "64"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "points/s"
    assert d["higher_is_better"] is True and d["config"]["workload"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_gpu_arm_refuses_to_run_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run(["--steps", "1", "--warmup", "0", "--no-extras"], timeout=120)
    assert r.returncode != 0
    assert "CUDA" in (r.stderr + r.stdout)


def test_binding_fails_loudly_without_the_library():
    """hc.load raises when libhc.so is absent (no CPU fallback exists)."""
    code = ("from paper_1109_0545_gb300 import build, hc\n"
            "build.SO = '/nonexistent/libhc.so'\n"
            "hc.load(build_if_missing=False)\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "libhc.so not built" in r.stderr


def test_compact_summary_is_small_and_keeps_the_comparisons():
    """The main JSON line carries a compact summary of the secondary measurements (the
    driver keeps only the end of the output): under 2.5 KB, with the equal-batching
    ratio of the mixed-precision tracker against the all-DD one."""
    sys.path.insert(0, ROOT)
    import bench
    fam = {"paths": 2432, "stage_cap": 200,
           "plain_one_path_per_launch": {"path_steps_per_s": 87.0, "paths_per_s": 0.4, "sample_paths": 16},
           "batched_all_dd_secant": {"path_steps_per_s": 34488.0, "paths_per_s": 170.0, "ok_paths": 0}}
    for v in ("batched_secant", "batched_quadratic", "batched_tangent", "batched_quadratic_proposer"):
        fam[v] = {"path_steps_per_s": 55539.0, "paths_per_s": 270.0, "ok_paths": 0,
                  "same_end_point_as_batched_all_dd_1e-28": 0, "status_hist": [0] * 7}
    reg = {k: (dict(v) if isinstance(v, dict) else v) for k, v in fam.items()}
    ex = {"tracker": {"uneven": fam, "uneven_regular": reg},
          "large_path_qd_n96": {"status": "MIN_STEP", "stages": 1937, "seconds": 30.9, "stages_per_s": 62.7,
                                "t_end": 0.99999986, "n": 96},
          "single_path_n8": {"n": 8, "monomials": 104, "plain_all_dd_secant": {"path_steps_per_s": 2254.0},
                             "fp64_refine_quadratic": {"path_steps_per_s": 3562.0}},
          "paper_tables": {"table4_dim40_deg2_qd": {"one_block": {"seconds": 1.3}, "whole_gpu": {"seconds": 0.5},
                                                    "paper_8_cores_s": 62.257}},
          "common_support_table1": {"per_term": {"eval_points_per_s": 42595.0}, "shared": {"eval_points_per_s": 61020.0}},
          "quality_up": {"quality_up_8_gpus": 1.85}, "eval_jac_points_per_s": 201926.0}
    c = bench.compact_extras(ex)
    assert len(json.dumps(c)) < 2500
    assert abs(c["tracker_uneven"]["mixed_vs_all_dd_equal_batching"] - 55539.0 / 34488.0) < 1e-2
    assert c["tracker_uneven"]["plain_sample_paths"] == 16
    assert c["large_path_qd_n96"]["stages"] == 1937
