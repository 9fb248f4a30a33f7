"""The reference arm of bench.py (`--impl reference`: the oracle as it stands, timed on
the host cores) prints the same JSON line as the CUDA arm, marked impl = reference, with
its own cpu_baseline and an e2e block that moves no bytes; its solve reaches the
tolerance.  Runs on the CPU (the arm needs no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "0", "--workload", "q1_poisson_64x64"],
                         cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "solves/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "q1_poisson_64x64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["relres_max"] <= 1e-10


def test_l2_note_states_the_working_set_against_l2():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    big = bench.l2_note(121e6, 615e6, 525e6, 129e6)  # the 1024^2 step: CSR, factor, fronts
    assert big.startswith("inputs larger than L2") and "1261 MB" in big and "129 MB" in big
    small = bench.l2_note(0.4e6, 3e6, 4e6, 129e6)   # the 64^2 step fits in L2
    assert small.startswith("working set 7 MB, within the 129 MB L2")
