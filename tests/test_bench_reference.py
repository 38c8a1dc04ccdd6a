"""bench.py --impl reference on CPU: the FP64 oracle timed on the host cores prints the same JSON
line as the GPU arm (metric, unit, direction, config), with impl, cpu_baseline and a zero-copy e2e,
on the configuration the command line names (--iters applies to both arms)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*argv):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *argv],
                       capture_output=True, text=True, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("iters,cpu_iters,sampled", [(4, 2, 2), (2, 20, 2), (0, 20, 0)])
def test_reference_line(iters, cpu_iters, sampled):
    d = _run("--workload", "c1", "--steps", "1", "--warmup", "0", "--iters", str(iters),
             "--cpu-iters", str(cpu_iters))
    assert d["impl"] == "reference"
    assert d["metric"] == "ms per PDF reconstruction" and d["unit"] == "ms"
    assert d["higher_is_better"] is False and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["ms_per_step"] == d["value"]
    assert d["config"]["iters"] == iters and d["config"]["workload"].startswith("c1:")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert f"{sampled} Adam iterations" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
