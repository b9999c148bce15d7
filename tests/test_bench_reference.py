"""The benchmark's reference arm (the oracle timed on the host cores) prints
one JSON line with the contract's keys, on a short sample; no GPU needed."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def reference_line(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "3",
           "--cpu-seconds", "1", *extra]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("extra", [("--workload", "lfr-100k"),
                                   ("--workload", "uneven-batch", "--batch-graphs", "6",
                                    "--batch-node-scale", "0.03")])
def test_reference_arm_line(extra):
    d = reference_line(*extra)
    assert d["impl"] == "reference"
    assert d["metric"] == "seed expansions/s" and d["unit"] == "units/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"] and d["data"] == "synthetic"


def test_reference_arm_unavailable_workload():
    d = reference_line("--workload", "accuracy")
    assert d["impl"] == "reference" and "unavailable" in d


def test_reference_arm_never_loads_the_product_library():
    """The reference arm is the oracle alone: after it has run, no module of
    the CUDA binding is imported and libmscd.so is not mapped."""
    code = ("import sys, json; sys.argv = ['bench.py', '--impl', 'reference', '--steps', '1', '--warmup', '3', "
            "'--cpu-seconds', '1', '--workload', 'lfr-100k']; import bench; bench.main(); "
            "maps = open('/proc/self/maps').read(); "
            "print(json.dumps({'mscd_imported': 'paper_1301_0955_gb300.mscd' in sys.modules, "
            "'libmscd_mapped': 'libmscd' in maps, 'liborc_mapped': 'liborc' in maps}))")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    probe = lines[-1]
    assert lines[0]["impl"] == "reference"
    assert probe == {"mscd_imported": False, "libmscd_mapped": False, "liborc_mapped": True}
