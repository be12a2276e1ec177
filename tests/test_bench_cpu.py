"""The benchmark's CPU legs (no GPU): the reference arm's JSON line and the bounded,
extrapolated oracle sample it is built on."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line_on_tiny_workload():
    """`bench.py --impl reference` prints one JSON line on the workload's own explicit
    contour, with the step time it measured and the fraction of an apply per step."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "4^4-fp64-nq32-1src", "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "applies/s"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    # value = applies covered per step / step time
    assert abs(line["value"] * line["ms_per_step"] / 1e3 - line["applies_per_step"]) <= 1e-9 + 1e-6 * line[
        "applies_per_step"]
    c = line["config"]["contour"]
    assert (c["gamma"], c["rho"], c["alpha"], c["n_q"]) == (3.36, 3.36, 0.25, 32)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["host_cpu_count"] >= 1
    assert len(cb["extrapolated_iterations_per_node"]) == cb["sampled_nodes"]


def test_oracle_sample_extrapolation():
    """The sample's work estimate: nodes that converge inside the cap count their own
    iterations; the others are extrapolated from their residual reduction, and the
    sampled nodes are scaled to all of them."""
    sys.path.insert(0, ROOT)
    import bench
    import synthetic as S
    from oracle import contour

    dims = (2, 2, 2, 4)
    U = S.su3_links(dims, 0.5, 1401)
    b = S.gaussian_spinor(dims, 1402)
    z, c, c0 = contour.single_contour(8, 3.36, 3.36, 0.25)
    full = bench.OracleSample(U, b, z, c, c0, 100000)
    assert all(x < 100000 for x in full.need)  # every sampled node converged
    capped = bench.OracleSample(U, b, z, c, c0, 5)
    assert all(n >= 5 for n in capped.need)
    # the extrapolated counts land within a factor of a few of the converged ones
    ratio = np.array(capped.need) / np.array(full.need)
    assert np.all(ratio > 0.2) and np.all(ratio < 5.0)
    assert capped.work == sum(capped.need) * len(z) / len(capped.idx)
