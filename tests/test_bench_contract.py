"""The benchmark's contract on the CPU: the reference arm (the FP64 oracle)
prints its JSON line, and the DRAM-traffic figure is reported only for the
kernel sources it was taken on."""
import json
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def test_reference_arm_prints_its_line():
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--steps", "1", "--warmup",
                          "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["value"] > 0 and line["unit"] == "Gbit/s" and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in line["config"]


def test_traffic_is_reported_only_for_the_recorded_kernel_sources(tmp_path, monkeypatch):
    sys.path.insert(0, str(ROOT))
    import bench

    monkeypatch.setattr(bench, "PROFILE_DIR", tmp_path)
    assert bench.recorded_traffic("f32") == (None, None)
    page = "# summary\n\n- source_hash: `{h}`\n- dram_bytes_per_pass: 711434752\n"
    (tmp_path / "pass_kernels_n64800_f256_f32.md").write_text(page.format(h=bench.hot_source_hash()))
    traffic, src = bench.recorded_traffic("f32")
    assert traffic == pytest.approx(711434752.0) and src == "pass_kernels_n64800_f256_f32.md"
    (tmp_path / "pass_kernels_n64800_f256_f32.md").write_text(page.format(h="0123456789abcdef"))
    traffic, src = bench.recorded_traffic("f32")
    assert traffic is None and "stale" in src


@pytest.mark.gpu
def test_our_arm_prints_every_record():
    """A short run of the GPU arm: one JSON line with the timed steps, the
    pass roofline against the measured peak, the other message formats, the
    end-to-end figures, the early-exit form, the clocks, the launch count and
    the mixed-batch and serving records."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--steps", "5", "--warmup", "3", "--by-msg-steps", "5",
                          "--early-exit-steps", "1", "--e2e-steps", "2", "--no-cpu-baseline", "--serve-requests", "200"],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks", "by_msg",
                "early_exit_max_iter_50", "mixed_batch", "serving"):
        assert key in line, key
    assert line["value"] > 0 and line["gpu_launches"] > 0 and line["steps"] == 5
    rl = line["roofline"]
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s" and rl["frac"] == pytest.approx(rl["achieved"] / rl["peak"])
    assert set(line["by_msg"]) == {"f32", "f16", "bf16", "i8"}
    assert line["e2e"]["h2d_bytes_per_step"] > 0 and line["e2e"]["value"] > 0
    assert {r["rate_req_s"] for r in line["serving"]} == {2000.0, 10000.0, 50000.0}
    assert line["mixed_batch"]["batch_graph_f32"]["ms"] > 0
