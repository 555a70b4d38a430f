"""The benchmark's reference arm (the FP64 oracle on the host cores) runs on
the CPU and prints the one-line JSON record the measurement contract asks
for; the kernel-source hash that keys the recorded ncu traffic covers the
evaluation sources and changes when one of them does."""
import json
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "cubic16",
                        "--steps", "2", "--warmup", "1"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    # the GPU arm prints the same metric and unit strings (one constant each)
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["cpu_baseline"]["unit"] == bench.UNIT and d["e2e"]["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "cubic16",
                        "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_kernel_hash_tracks_the_evaluation_sources(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    h0 = bench.kernel_hash()
    assert len(h0) == 16
    # a copy of the sources with one kernel file changed hashes differently
    import shutil
    root = tmp_path / "repo"
    shutil.copytree(os.path.join(ROOT, "paper_1204_1121_gb300", "csrc"),
                    root / "paper_1204_1121_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.kernel_hash() == h0
    f = root / "paper_1204_1121_gb300" / "csrc" / "blip_staged.cu"
    text = f.read_text()
    f.write_text(text + "\n// a comment and more blank space\n\n")
    assert bench.kernel_hash() == h0                   # comments do not count
    f.write_text(text + "\nstatic int unused_probe;\n")
    assert bench.kernel_hash() != h0                   # code does
    f.write_text(text)
    # the Sherman-Morrison update and the fused-ratio kernels are not part of
    # the evaluation path
    for name in ("blip_sm.cu", "blip_ratio.cu", "blip_ratio_tc.cu"):
        g = root / "paper_1204_1121_gb300" / "csrc" / name
        g.write_text(g.read_text() + "\nstatic int unused_probe;\n")
        assert bench.kernel_hash() == h0
    # the helpers the tensor-core evaluation kernel shares with the ratio
    # kernel are
    g = root / "paper_1204_1121_gb300" / "csrc" / "blip_tc_common.cuh"
    g.write_text(g.read_text() + "\nstatic int unused_probe;\n")
    assert bench.kernel_hash() != h0
