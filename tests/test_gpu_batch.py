"""Batched stepping (ml_batch_*) of several independent grids of uneven size and
content: the results are bit-identical to stepping each grid alone with ml_step
(fields, density matrices, DFT sums, absorbed energy), for every field-pass grid
shape and with or without the captured graph; the autotuner leaves the state as it
found it.
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


def problems():
    return [
        W.small_coupled(0, shape=(37, 22, 29), nmol=6, drude=True),
        W.small_coupled(1, shape=(24, 20, 28), nmol=0, source=True),
        W.small_coupled(2, shape=(40, 17, 33), nmol=9, periodic=(True, False, False)),
        W.small_coupled(3, shape=(19, 26, 21), nmol=3, eps_map=False, planes=False),
        W.small_coupled(4, shape=(33, 33, 18), nmol=5, drude=True, periodic=(False, True, True)),
        W.small_coupled(5, shape=(29, 27, 31), nmol=4, drude=True, lorentz=True, eps_map=False),
    ]


def state(ml, g, prob):
    out = {"fields": g.fields(), "absorbed": g.absorbed(), "flux": [g.plane_data(p) for p in range(len(prob.planes))]}
    if prob.molecules.count:
        out["rho"] = g.molecules(ml.ML_MOL_RHO)
    return out


def same(a, b):
    for x, y in zip(a["fields"], b["fields"]):
        assert np.array_equal(x, y)
    assert a["absorbed"] == b["absorbed"]
    for pa, pb in zip(a["flux"], b["flux"]):
        for x, y in zip(pa, pb):
            assert np.array_equal(x, y)
    if "rho" in a:
        assert np.array_equal(a["rho"], b["rho"])


def run_single(ml, probs, precision, steps):
    out = []
    for p in probs:
        g = ml.Grid(p, precision)
        try:
            g.step(steps)
            out.append(state(ml, g, p))
        finally:
            g.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("tuning", [(3, True), (1, True), (0, True), (2, False)])
def test_batch_matches_single_grids(ml, precision, tuning):
    if precision == 1 and tuning[0] > 1:
        pytest.skip("FP64 field pass holds one block per SM")
    probs = problems()
    steps = 134  # two captured 64-step sequences and a 6-step tail
    ref = run_single(ml, probs, precision, steps)
    grids = [ml.Grid(p, precision) for p in probs]
    try:
        b = ml.Batch(grids)
        b.tune(*tuning)
        b.step(steps)
        for g, p, r in zip(grids, probs, ref):
            assert g.nstep == steps
            same(state(ml, g, p), r)
        b.close()
    finally:
        for g in grids:
            g.close()


def test_batch_in_pieces_and_then_single(ml):
    """40 batched steps, 30 more, then 10 with ml_step: the fields and density
    matrices are those of 80 single steps (the DFT sums are grouped differently,
    so they agree to round-off)."""
    probs = problems()[:3]
    ref = run_single(ml, probs, 0, 80)
    grids = [ml.Grid(p, 0) for p in probs]
    try:
        b = ml.Batch(grids)
        b.step(40)
        b.step(30)
        for g in grids:
            g.step(10)
        for g, p, r in zip(grids, probs, ref):
            s = state(ml, g, p)
            for x, y in zip(s["fields"], r["fields"]):
                assert np.array_equal(x, y)
            if "rho" in r:
                assert np.array_equal(s["rho"], r["rho"])
            for pa, pb in zip(s["flux"], r["flux"]):
                for x, y in zip(pa, pb):
                    assert np.allclose(x, y, rtol=1e-5, atol=1e-6 * np.abs(y).max())
        b.close()
    finally:
        for g in grids:
            g.close()


def test_autotune_restores_state(ml):
    probs = problems()[:4]
    grids = [ml.Grid(p, 0) for p in probs]
    try:
        for g in grids:
            g.step(5)
        before = [state(ml, g, p) for g, p in zip(grids, probs)]
        b = ml.Batch(grids)
        choice, ms = b.autotune(32)
        assert choice in (0, 1, 2, 3) and ms > 0
        for g, p, r in zip(grids, probs, before):
            assert g.nstep == 5
            same(state(ml, g, p), r)
        b.step(33)
        b.close()
        ref = run_single(ml, probs, 0, 38)
        for g, p, r in zip(grids, probs, ref):
            s = state(ml, g, p)
            for x, y in zip(s["fields"], r["fields"]):
                assert np.array_equal(x, y)
    finally:
        for g in grids:
            g.close()


def test_energy_transfer_batch_matches_single_grids(ml):
    """Donor-acceptor realisations (two-, four- and eight-level acceptors at several
    distances), batched: bit-identical to stepping each grid alone."""
    probs = W.energy_transfer_batch(count=5, edge=48)
    steps = 70
    ref = run_single(ml, probs, 0, steps)
    grids = [ml.Grid(p, 0) for p in probs]
    try:
        b = ml.Batch(grids)
        b.step(steps)
        for g, p, r in zip(grids, probs, ref):
            same(state(ml, g, p), r)
        b.close()
    finally:
        for g in grids:
            g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_chunk_length_does_not_change_the_results(ml, precision):
    """The z-chunk length of the field pass (automatic, 2, 5, 16 planes) changes the
    blocks, not the arithmetic of a cell: fields and density matrices are bit-identical;
    the absorbed energy, summed per block, agrees to rounding."""
    base = W.small_coupled(0, shape=(37, 22, 29), nmol=6, drude=True, lorentz=True)
    out = []
    for z in (0, 2, 5, 16):
        g = ml.Grid(base.replace(zchunk=z), precision)
        try:
            g.step(45)
            out.append(state(ml, g, base))
        finally:
            g.close()
    for o in out[1:]:
        for x, y in zip(o["fields"], out[0]["fields"]):
            assert np.array_equal(x, y)
        assert np.array_equal(o["rho"], out[0]["rho"])
        assert abs(o["absorbed"] - out[0]["absorbed"]) <= (1e-12 if precision else 1e-5) * abs(out[0]["absorbed"])


@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, 1e-4)])
def test_batched_instances_against_oracle(ml, oracle_mod, precision, tol):
    """Every instance of a batch, stepped together through the graph-replayed launches,
    against the FP64 oracle stepping that instance alone: fields, density matrices,
    flux spectra and absorbed energy (relative L2; FP64 to round-off, FP32 within 1e-4)."""
    probs = [problems()[q] for q in (0, 2, 5)] + [W.plasmonic_instance(40, 30, np.random.default_rng(3), width=6.0)]
    grids = [ml.Grid(p, precision) for p in probs]
    b = ml.Batch(grids)
    try:
        b.step(110)  # one graph sequence of 64 steps and a remainder
        for g, p in zip(grids, probs):
            o = oracle_mod.OracleSim(p)
            o.step(110)
            fo = o.fields()
            scale = max(np.linalg.norm(f) for f in fo)
            for got, want in zip(g.fields(), fo):
                assert np.linalg.norm(np.asarray(got, np.float64) - want) < tol * scale
            M = p.molecules.count
            if M:
                rg = np.concatenate([g.rho(m).ravel() for m in range(M)])
                ro = np.concatenate([o.rho(m).ravel() for m in range(M)])
                assert np.linalg.norm(rg - ro) < tol * np.linalg.norm(ro)
            for q in range(len(p.planes)):
                fg, fw = g.flux(q), o.flux(q)
                assert np.abs(fg - fw).max() <= tol * max(np.abs(fw).max(), 1e-300)
            ab_o = o.absorbed()
            assert abs(g.absorbed() - ab_o) <= tol * max(abs(ab_o), 1e-300)
    finally:
        b.close()
        for g in grids:
            g.close()


def test_batch_tracing_counts_and_results(ml):
    """ml_batch_set_timing: traced steps run without the graph, one event pair per launch
    and kernel class, and give the same bits as untraced steps."""
    probs = [problems()[q] for q in (0, 2)]
    outs = []
    for traced in (False, True):
        grids = [ml.Grid(p, 0) for p in probs]
        b = ml.Batch(grids)
        try:
            if traced:
                ml.ml_batch_set_timing(b.h, True)
            b.step(70)
            if traced:
                ms, cnt = ml.ml_batch_timing(b.h)
                assert cnt[0] == 70 and cnt[4] == 70 and cnt[1] == 70  # molecules, current, field pass
                assert cnt[3] == 2  # folds: one full 64-step period and the tail
                assert np.all(ms[[0, 1, 3, 4]] > 0)
                ml.ml_batch_set_timing(b.h, False)
            outs.append([state(ml, g, p) for g, p in zip(grids, probs)])
        finally:
            b.close()
            for g in grids:
                g.close()
    for x, y in zip(outs[0], outs[1]):
        same(x, y)
