"""bench.py's reference arm (the FP64 oracle timed on the host cores) runs
without a GPU: one bounded step prints one JSON line with the contract's keys,
on the same metric and workload as the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line(tmp_path):
    rec = tmp_path / "runs.jsonl"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--record", str(rec)], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference"
    assert d["metric"] == "KK frames/s" and d["unit"] == "frames/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "L128_N75_T2048_i16_grid512x512_pairs75x128"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # --record appended one JSONL run record of the same run
    lines = rec.read_text().splitlines()
    assert len(lines) == 1
    rr = json.loads(lines[0])
    assert rr["impl"] == "reference" and rr["value"] == d["value"] and rr["workload"] == d["config"]["workload"]
    assert rr["host_cores"] == cb["cores"] and rr["argv"][-2:] == ["--record", str(rec)]


def test_run_record_of_a_gpu_line(tmp_path):
    """run_record keeps the contract's figures of a GPU-arm line (here a
    hand-made one) and leaves what the run did not measure null."""
    sys.path.insert(0, ROOT)
    import bench
    out = {"metric": "KK frames/s", "value": 580.0, "unit": "frames/s", "ms_per_step": 1.72, "n_gpus": 1,
           "config": {"workload": "W", "form": "chosen: BF16"},
           "e2e": {"value": 575.0}, "clocks": {"sm_mhz": 2070.0},
           "roofline": {"kernel": "k", "bound": "alu", "frac": 0.64, "achieved": 1.0},
           "breakdown": {"gpixel_pairs_per_s": 1600.0, "forms": {"bf16": {"frames_per_s": 580.0},
                                                                 "f32": {"frames_per_s": 507.0}}},
           "cpu_baseline": {"value": 0.4, "cores": 16, "gpu_rel_l2_vs_oracle_whole_image": {"bf16": 1e-3},
                            "gpu_wire_peaks_at_oracle_pixel": {"wires": 20, "exact": {"bf16": 20}}}}
    rr = bench.run_record(out, argv=["--steps", "3"])
    assert rr["value"] == 580.0 and rr["e2e"] == 575.0 and rr["workload"] == "W" and rr["seed"] == 2000
    assert rr["frames_per_s_by_form"] == {"bf16": 580.0, "f32": 507.0}
    assert rr["rel_l2_vs_oracle"] == {"bf16": 1e-3} and rr["wire_peaks_at_oracle_pixel"]["exact"]["bf16"] == 20
    assert rr["roofline"] == {"kernel": "k", "bound": "alu", "frac": 0.64} and rr["host_cores"] == 16
    bench.append_record(str(tmp_path / "r.jsonl"), rr)
    bench.append_record(str(tmp_path / "r.jsonl"), bench.run_record({"value": 1.0}, argv=[]))
    lines = (tmp_path / "r.jsonl").read_text().splitlines()
    assert len(lines) == 2 and json.loads(lines[1])["roofline"] is None


def test_refiner_per_layer_bound_limits():
    """The per-layer roofline bound reduces to the FLOP count over the peak
    when bandwidth is unlimited, and exceeds each single-resource bound
    otherwise."""
    sys.path.insert(0, ROOT)
    import bench
    fwd_flops, step_flops = bench.refiner_conv_flops(16)
    f_inf, s_inf = bench.refiner_conv_attainable_ms(16, 1e12, 1000.0)      # effectively unlimited HBM
    assert abs(f_inf - fwd_flops / 1e15 * 1e3) / f_inf < 1e-6
    assert abs(s_inf - step_flops / 1e15 * 1e3) / s_inf < 1e-6
    f, s = bench.refiner_conv_attainable_ms(16, 6697.0, 1910.7)
    assert f > fwd_flops / 1910.7e12 * 1e3 and s > step_flops / 1910.7e12 * 1e3
    assert s > 2 * f
