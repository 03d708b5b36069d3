"""Host-side parts of the benchmark's contract, without a GPU: the reference arm's JSON line and
the rule that a stored DRAM-traffic figure is used only on the sources it was captured on."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_only_on_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.txt").write_text(json.dumps(
        {"me_kernel:ggttgg": {"source_sha": "abc", "dram_bytes_per_event": 5.0}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_source_sha", lambda: "abc")
    assert bench._traffic_per_event("me_kernel", "ggttgg") == 5.0
    assert bench._traffic_per_event("me_kernel_float", "ggttgg") is None
    monkeypatch.setattr(bench, "_source_sha", lambda: "def")
    assert bench._traffic_per_event("me_kernel", "ggttgg") is None


def test_source_hash_covers_the_cuda_sources():
    h = bench._source_sha()
    assert len(h) == 16 and h == bench._source_sha()


def test_reference_arm_line():
    """`bench.py --impl reference` times the oracle on the host cores and prints one JSON line with
    the keys of the contract (no GPU, no torch.cuda)."""
    env = dict(os.environ, OMP_NUM_THREADS="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "events/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("g g > t t~ g g")
    # the GPU arm's default line carries exactly this config, so the two arms compare like for like
    assert line["config"] == bench._workload_config(bench.NEVT, "fp64", "ggttgg")
