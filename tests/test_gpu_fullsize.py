"""The benchmarked workload at its full size and in the launch configuration bench.py
times (FP32, molecule -> current -> field pass as programmatic dependent launches):

- against the FP64 oracle: the 256^3 superradiant slab with 10,000 two-level emitters,
  20 steps from seeded random fields, every field value (relative L2 <= 1e-4) and every
  emitter's populations;
- the overlapped launch chain against the serialised one (ML_PDL=0, read when a grid is
  created) on a 128^3 copy: bit-identical fields, density matrices and DFT sums.  A
  dependency the overlap had lost would show up here as a difference.
"""
import numpy as np
import pytest

from paper_2512_06173_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ml():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2512_06173_gb300 import maxlink
    maxlink.load()
    return maxlink


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def random_fields(prob, seed):
    """Seeded unit-variance fields, rounded to FP32 so that both sides start equal."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((prob.nz, prob.ny, prob.nx)).astype(np.float32).astype(np.float64)
            for _ in range(6)]


def run(ml, prob, steps, fields):
    g = ml.Grid(prob, 0)
    try:
        g.set_fields(fields)
        g.step(steps)
        g.sync()
        return g.fields(), g.molecules(ml.ML_MOL_RHO), [g.plane_data(p) for p in range(len(prob.planes))]
    finally:
        g.close()


def test_overlapped_chain_is_bit_identical_to_serialised(ml, monkeypatch):
    prob = W.superradiant_slab(n=128, nmol=3000)
    f0 = random_fields(prob, 1)
    monkeypatch.setenv("ML_PDL", "0")
    ref = run(ml, prob, 80, f0)
    monkeypatch.setenv("ML_PDL", "1")
    got = run(ml, prob, 80, f0)
    for x, y in zip(got[0], ref[0]):
        assert np.array_equal(x, y)
    assert np.array_equal(got[1], ref[1])
    for pa, pb in zip(got[2], ref[2]):
        for x, y in zip(pa, pb):
            assert np.array_equal(x, y)


def test_full_size_bench_workload_against_oracle(ml, oracle_mod):
    prob = W.superradiant_slab()
    f0 = random_fields(prob, 2)
    steps = 20
    g = ml.Grid(prob, 0)
    try:
        g.set_fields(f0)
        g.step(steps)
        g.sync()
        fg = g.fields()
        pops = g.molecules(ml.ML_MOL_POP)
    finally:
        g.close()
    o = oracle_mod.OracleSim(prob)
    o.set_fields(f0)
    o.step(steps)
    for got, want in zip(fg, o.fields()):
        assert rel(got, want) < 1e-4
    po = np.array([np.real(p[:2]) for p in o.populations()])
    assert np.abs(pops[:, :2] - po).max() < 1e-4
