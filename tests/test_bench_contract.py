"""bench.py's reference arm (the CPU oracle timed on the host cores) on the CPU: it prints one
JSON line with the fields the benchmark contract names, and under a multi-rank launch only rank
0 runs it (the others exit 0 without work or output).  The small-memory case keeps the run to a
few seconds: it renders 32 frames instead of 300, and one timed step is one room frame.  Also
the rule that ties the reported fusion DRAM traffic to the kernels' source."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CMD = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
       "--small-memory"]


def run(env_extra):
    env = dict(os.environ, **env_extra)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    return subprocess.run(CMD, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    p = run({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "frames/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["data"] == "synthetic" and isinstance(d["config"]["workload"], str)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert isinstance(cb["sample"], str) and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_zero_only():
    p = run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_fusion_traffic_follows_the_device_code(tmp_path, monkeypatch):
    """The ncu-derived DRAM traffic is reported only while the committed summary's hash equals
    the hash of frame.cu's device code: an edit after the kernels' namespace (host launchers)
    keeps it, an edit inside it makes it None."""
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "paper_1805_03709_b300", "csrc", "frame.cu")) as f:
        src = f.read()
    # a summary taken from the current kernels (the committed one may predate a kernel edit)
    digest = bench.device_source_digest(
        os.path.join(ROOT, "paper_1805_03709_b300", "csrc", "frame.cu"))
    prof = (f"device_source_sha256_16: {digest}\n"
            "dram_bytes_per_touched_block: 4640\n")
    fake = tmp_path / "repo"
    (fake / "paper_1805_03709_b300" / "csrc").mkdir(parents=True)
    (fake / "profiles").mkdir()
    (fake / "profiles" / "k_integrate_room_640x480.txt").write_text(prof)
    cu = fake / "paper_1805_03709_b300" / "csrc" / "frame.cu"
    monkeypatch.setattr(bench, "ROOT", str(fake))
    cu.write_text(src)
    per_block = bench.profile_traffic(1.0)
    assert per_block is not None and per_block > 0
    assert bench.profile_traffic(1000.0) == 1000.0 * per_block
    cu.write_text(src + "\n// a host-side edit after the kernels\n")
    assert bench.profile_traffic(1.0) == per_block
    cu.write_text(src.replace("namespace {", "namespace {\n// an edit among the kernels", 1))
    assert bench.profile_traffic(1.0) is None
