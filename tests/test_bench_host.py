"""Host-side arithmetic of bench.py that the reported roofline rests on: the
algorithmic bytes of one field-pass launch, checked against hand counts."""
import os
import sys

import numpy as np

from paper_2512_06173_gb300.workloads import Material, Problem

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_vacuum_and_cpml_bytes():
    # E and H read and written: 12 values per cell
    assert bench.field_pass_bytes(Problem(10, 12, 14, 0.5), 4) == 48 * 10 * 12 * 14
    assert bench.field_pass_bytes(Problem(10, 12, 14, 0.5), 8) == 96 * 10 * 12 * 14
    # four CPML memories read and written per cell and layer axis: 2 + 3 x-layers on a
    # 10-wide grid cover 5 of its 10 columns, the 4 z-layers 4 of 14 planes
    p = Problem(10, 12, 14, 0.5, pml=(2, 3, 0, 0, 4, 0))
    N = 10 * 12 * 14
    assert bench.field_pass_bytes(p, 4) == 48 * N + 32 * (5 * 12 * 14) + 32 * (10 * 12 * 4)


def test_material_and_pole_bytes():
    n = 6
    mat = np.zeros((n, n, n), np.uint8)
    mat[0] = 1  # 36 Drude cells
    mat[1] = 2  # 36 Lorentz cells
    mat[2] = 3  # 36 cells with a Drude and two Lorentz poles
    mats = [Material(1.0), Material(1.0, 1.0, 0.1), Material(2.0, 0.5, 0.1, 0.4),
            Material(1.0, 0.7, 0.1, extra=((0.3, 0.1, 0.5), (0.2, 0.05, 0.9)))]
    p = Problem(n, n, n, 0.5, mat=mat, materials=mats)
    N = n ** 3
    # per pole 6 values for J (3 read + 3 written), per Lorentz pole 6 more for P
    want = 48 * N + N + 36 * (24) + 36 * (24 + 24) + 36 * (3 * 24 + 2 * 24)
    assert bench.field_pass_bytes(p, 4) == want
    # a design box adds one coefficient per cell
    q = Problem(n, n, n, 0.5, design_box=(1, 1, 1, 2, 3, 4), design_eps=np.ones((4, 3, 2)))
    assert bench.field_pass_bytes(q, 4) == 48 * N + 4 * 24


def bench_args(argv):
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--bragg-shape", type=int, nargs=3, default=(512, 512, 384))
    ap.add_argument("--bragg-nmol", type=int, default=100000)
    return ap.parse_args(argv)


def test_headline_config_is_the_bragg_ensemble():
    """The line's workload is the 512 x 512 x 384 Bragg-resonator ensemble with 100,000
    multilevel systems (the largest single-GPU configuration)."""
    args = bench_args([])
    prob = bench.headline_problem(args)
    c = bench.config_of(prob, 1)
    assert c["grid"] == [512, 512, 384] and c["molecules"] == 100000 and c["cells"] == 512 * 512 * 384
    assert "Bragg" in c["workload"] and "100000" in c["workload"]
    nl = prob.molecules.nlev
    assert nl.min() == 2 and nl.max() == 8


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints one JSON line
    with the keys the contract asks for; run here on a small cube for speed."""
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--bragg-shape", "96",
                        "48", "40", "--bragg-nmol", "40", "--steps", "2", "--warmup", "1", "--ref-budget", "2"],
                       capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["value"] > 0 and d["unit"] == "Gcell-updates/s" and d["steps"] >= 1 and d["warmup"] == 3  # W >= 3 is enforced
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "96x48x40" in cb["sample"]
    # the same config object as the CUDA arm's line for the same arguments
    args = bench_args(["--bragg-shape", "96", "48", "40", "--bragg-nmol", "40"])
    assert d["config"] == json.loads(json.dumps(bench.config_of(bench.headline_problem(args), 1)))
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
