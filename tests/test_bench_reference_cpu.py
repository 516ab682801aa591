"""The benchmark's reference arm on the host: the oracle evaluates a bounded sample of an
amplitude's slice terms per step and the script prints one JSON line with the contract's
keys. Run on small workloads so it ends in seconds."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("args,sliced", [(("--workload", "grid4x4d10"), 0),
                                          (("--workload", "grid6x6d25-k12", "--sliced", "4", "--plan-trials", "4",
                                            "--circuit-seed", "2003"), 4)])
def test_reference_arm_prints_one_contract_line(args, sliced):
    d = _run("--steps", "1", "--warmup", "0", *args)
    assert d["impl"] == "reference" and d["unit"] == "amplitudes/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["config"]["sliced"] == sliced
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "amplitudes/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
