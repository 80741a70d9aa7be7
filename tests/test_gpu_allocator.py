"""The boundary's allocator callback (ml_set_allocator).

The Python binding installs an allocator backed by PyTorch's caching allocator when it
loads the library, so every device buffer of a grid, a batch and an adjoint call comes
from PyTorch (the step itself allocates nothing).  These tests count the callback's
calls, check that everything allocated is returned, that PyTorch sees the memory, and
that results do not depend on the allocator (the library's default is cudaMallocAsync).
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
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_grid_memory_comes_from_torch(ml, oracle_mod):
    import torch
    al = ml.use_torch_allocator()
    assert ml.allocator() is al
    n0, f0, live0 = al.allocs, al.frees, al.live_bytes
    torch.cuda.synchronize()
    t0 = torch.cuda.memory_allocated()
    prob = W.small_coupled(seed=2, shape=(39, 22, 29))
    g = ml.Grid(prob, 0)
    try:
        made = al.allocs - n0
        assert made >= 20  # fields, CPML, tables, molecules, planes ...
        held = al.live_bytes - live0
        assert held >= 12 * g.prob.cells * 4  # two levels of six FP32 field arrays at least
        assert torch.cuda.memory_allocated() - t0 >= held
        s0 = al.allocs
        g.step(30)
        g.sync()
        assert al.allocs == s0  # stepping allocates nothing
        o = oracle_mod.OracleSim(prob)
        o.step(30)
        for a, b in zip(g.fields(), o.fields()):
            assert rel(a, b) < 1e-4
    finally:
        g.close()
    assert al.frees - f0 == al.allocs - n0
    assert al.live_bytes == live0


def test_batch_and_adjoint_memory_comes_from_torch(ml):
    al = ml.use_torch_allocator()
    probs = [W.small_coupled(seed=s, shape=(37 + s, 22, 29)) for s in range(3)]
    grids = [ml.Grid(p, 0) for p in probs]
    try:
        n0, live0 = al.allocs, al.live_bytes
        b = ml.Batch(grids)
        b.step(70)  # argument arrays, work lists, graph sequence
        assert al.allocs - n0 >= 5
        held = al.live_bytes - live0
        assert held > 0
        b.autotune(8)  # state snapshots for the trials, returned at the end of the call
        assert al.live_bytes - live0 == held
        b.close()
        assert al.live_bytes == live0
    finally:
        for g in grids:
            g.close()
    prob = W.adjoint_design(n=24, design=10, nmol=20, pml=4, sigma=1.0, width=6.0, mol_x=(8.0, 11.0), seed=14)
    g = ml.Grid(prob, 0)
    try:
        n0, live0 = al.allocs, al.live_bytes
        obj, ge, gg = g.adjoint(60, 0, 0, ckpt_every=20)
        assert al.allocs - n0 >= 10  # checkpoints, adjoint fields, records ...
        assert al.live_bytes == live0  # the call's work memory is returned
        assert np.isfinite(obj) and np.all(np.isfinite(ge)) and np.all(np.isfinite(gg))
    finally:
        g.close()


def test_default_allocator_gives_the_same_bits(ml):
    prob = W.small_coupled(seed=1, shape=(38, 22, 29))
    outs = []
    for use_torch in (True, False):
        if use_torch:
            ml.use_torch_allocator()
        else:
            ml.use_default_allocator()
        al = ml.allocator()
        n0 = al.allocs if al else None
        g = ml.Grid(prob, 0)
        try:
            g.step(40)
            outs.append((g.fields(), g.molecules(ml.ML_MOL_RHO)))
        finally:
            g.close()
        if al is None:
            assert ml.allocator() is None
        else:
            assert al.allocs > n0
    ml.use_torch_allocator()
    for x, y in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(x, y)
    assert np.array_equal(outs[0][1], outs[1][1])


def test_allocator_arguments(ml):
    import ctypes as C
    L = ml.load()
    a = ml.TorchAllocator()
    assert L.ml_set_allocator(a.c_alloc, ml._FREE_T(), None) == ml.ML_ERR_INVALID_ARG
    assert L.ml_set_allocator(ml._ALLOC_T(), a.c_free, None) == ml.ML_ERR_INVALID_ARG


def test_refused_allocation_gives_oom_and_returns_memory(ml, oracle_mod):
    """An allocator that refuses: grid creation fails with ML_ERR_OOM, every buffer the
    call had taken goes back through the callback, and the library keeps working."""
    ga = ml.use_torch_allocator()
    L = ml.load()
    al = ml.TorchAllocator()
    limit = 10

    def refusing(pp, nbytes, stream, ctx):
        if al.allocs >= limit:
            return 1
        return al._alloc(pp, nbytes, stream, ctx)

    c_alloc = ml._ALLOC_T(refusing)
    assert L.ml_set_allocator(c_alloc, al.c_free, None) == ml.ML_OK
    prob = W.small_coupled(seed=3, shape=(37, 22, 29))
    try:
        with pytest.raises(ml.MaxlinkError) as e:
            ml.Grid(prob, 0)
        assert e.value.status == ml.ML_ERR_OOM
        assert al.allocs == limit and al.frees == limit and al.live_bytes == 0
    finally:
        assert L.ml_set_allocator(ga.c_alloc, ga.c_free, None) == ml.ML_OK
    g = ml.Grid(prob, 0)
    try:
        g.step(20)
        g.sync()
        o = oracle_mod.OracleSim(prob)
        o.step(20)
        for a, b in zip(g.fields(), o.fields()):
            assert rel(a, b) < 1e-4
    finally:
        g.close()
