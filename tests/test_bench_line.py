"""bench.py's headline: the last stdout line must be one JSON object under
2 KB with the keys of the benchmark contract, however many rows, kernels and
autotuner entries the run measured (those go to the detail file)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _fake_run():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        precision = "bf16x3"
        steps = 20
        warmup = 5
        detail_file = "bench_detail.json"
    kernels = {f"kernel_{i}_with_a_long_template_name<{i}, true>":
               {"ms_per_launch": 0.1 * i, "launches": 20, "share": 0.05 * i} for i in range(14)}
    peaks = {"hbm_gbs": 6789.3, "bf16_tflops": 1911.8, "sm_max_mhz": 2070.0, "src": "measured"}
    roof = bench.roofline_for("cgemm_tc", 0.62, 426, peaks, 2070.0, "bf16x3")
    roof["kernel"] = "cgemm_tc"
    compare = [{"precision": "tf32x3", "ms_per_step": 2.4, "value": 131.0},
               {"precision": "fp32", "ms_per_step": 9.7, "value": 33.0}]
    errors = {"bf16x3": {"rel_err": 5.3e-6, "picks_equal": True},
              "tf32x3": {"rel_err": 6.1e-6, "picks_equal": True},
              "fp32": {"rel_err": 5.4e-7, "picks_equal": True}}
    rows = {f"row{i}": {"gpu_ms": 1.0 + i, "workload": "x" * 200, "cases": list(range(50))}
            for i in range(12)}
    rows["completion_batched"] = {"warm_iteration_ms": 80.0, "iterations": 100,
                                  "relative_error_to_truth": 0.01}
    rows["completion_batched_bf16x3"] = {"warm_iteration_ms": 81.0, "iterations": 25,
                                         "relative_error_to_truth": 0.02}
    rsvd = {"value": 300.0, "ms_per_tensor": 3.3, "unit": "tensors/s",
            "compare": {"fp32_tensors_per_s": 200.0, "rel_err": 1e-6, "fp32_rel_err": 1e-7},
            "cpu_baseline": {"value": 0.02}}
    e2e = {"value": 17.3, "unit": "TFLOP/s", "ms_per_step": 18.6,
           "h2d_bytes_per_step": 3584000000, "d2h_bytes_per_step": 768000000, "pipeline": "x"}
    cpu = {"value": 0.06, "unit": "TFLOP/s", "cores": 16, "kind": "oracle", "sample": "s" * 150}
    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 9}
    return bench.headline(Args(), 1, 168.5, 1.912, 426, 154, roof, kernels, cpu, e2e, clocks,
                          compare, errors, rsvd, rows, peaks)


def test_headline_is_short_and_complete():
    line = _fake_run()
    text = json.dumps(line)
    assert len(text) < 2048, len(text)
    back = json.loads(text)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert key in back, key
    assert "workload" in back["config"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in back["roofline"], key
    for key in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert key in back["e2e"], key
    for key in ("value", "unit", "cores", "kind", "sample"):
        assert key in back["cpu_baseline"], key
    # nominal work against the bf16 peak, and the executed split products beside it
    r = back["roofline"]
    assert abs(r["pipe_frac"] - 3 * r["frac"]) < 1e-3 * r["pipe_frac"]
    assert abs(r["achieved"] / r["peak"] - r["frac"]) < 1e-3


def test_step_bytes_of_the_workload():
    sys.path.insert(0, ROOT)
    import bench
    # A and B once (3.584 GB), the picks once, Z once (0.768 GB)
    b = bench.step_bytes(426)
    assert abs(b - (3.584e9 + 4 * 2000 * 426 * 64 + 4 * 426 * 1500 * 64 + 0.768e9)) < 1
