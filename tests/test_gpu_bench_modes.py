"""The benchmark's own GPU paths on a small workload (GPU): the default independent-source
mode and the node-sharded mode (contour nodes split over ranks; one rank here, so the
sum over ranks is the identity and the line must equal the plain sign apply's work)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "4^4-fp64-nq32-1src",
                        "--steps", "2", "--warmup", "1", "--no-e2e", "--no-cpu-baseline", *args],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])


def test_bench_sources_and_nodes_modes():
    a = _line()
    assert a["scaling"] == "weak" and a["value"] > 0 and a["solver"]["converged"] == 1
    assert a["gpu_launches"] > 0 and a["roofline"]["kernel"]
    b = _line("--parallel", "nodes")
    assert b["scaling"] == "strong" and b["value"] > 0 and b["solver"]["converged"] == 1
    assert "contour nodes split" in b["config"]["parallelism"]
