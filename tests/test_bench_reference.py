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


def test_traffic_records_are_tied_to_their_kernel_sources():
    """The DRAM traffic bench.py reports comes from profiles/*.json only while
    the hash of the kernel's sources matches the recorded one: the committed
    records match the committed sources, and any other source set (a changed
    kernel) yields no figure."""
    sys.path.insert(0, ROOT)
    import bench

    assert bench._traffic("f16", 512 ** 3) is not None
    assert bench._traffic("f32", 512 ** 3) is not None
    assert bench._md_traffic(200000) is not None
    assert bench._recorded("lb_step_traffic.json", "f16", ("lb_step.cu",)) is None
    assert bench._recorded("md_substep_traffic.json", "k_md_substep", ("md.cu",)) is None
