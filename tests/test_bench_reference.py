"""bench.py's reference arm (the oracle, on the host cores) runs without a
GPU and prints the contract's JSON line for the same metric and config as
the GPU arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "chain500_lattice32", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "coupled LB-MD MLUPS" and line["unit"] == "MLUPS" and line["higher_is_better"]
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    assert line["config"]["workload"] == "chain500_lattice32"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_traffic_records_are_tied_to_their_kernel_sources(tmp_path, monkeypatch):
    """The DRAM traffic bench.py reports comes from profiles/*.json only while
    the hash of the kernel's sources matches the recorded one: a record taken
    on one source is returned, and nothing once that source changes."""
    sys.path.insert(0, ROOT)
    import bench

    csrc = tmp_path / "paper_2305_05025_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_text("// kernel, first version\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"f16": {"kernel_hash": bench._kernel_hash(("k.cu",)), "dram_bytes_per_node": 72.7}}
    (tmp_path / "profiles" / "t.json").write_text(json.dumps(rec))
    assert bench._recorded("t.json", "f16", ("k.cu",))["dram_bytes_per_node"] == 72.7
    (csrc / "k.cu").write_text("// kernel, changed\n")
    assert bench._recorded("t.json", "f16", ("k.cu",)) is None
    assert bench._recorded("t.json", "f32", ("k.cu",)) is None
