"""The device status word (ml_sync_status) in the forms that fault nothing.

The paper's coupling hub detects failed or silent drivers with a barrier and timeouts
(Sec. III).  Here two device-side failures latch a status word that the host reads:

- ML_ERR_TIMEOUT: a field-pass block gives up on a bounded wait for a plane of its copy
  ring.  ml_set_wait_limit(g, 0) makes every such wait give up at once (no probe), so
  the timeout path runs without any wait being left pending: the blocks drain their own
  copies with the default bound and exit.
- ML_ERR_NUMERIC: a NaN in the field, written from the host with ml_set_fields, reaches
  a molecule's regularised field.

After either, the context stays usable: the same process then runs a small coupled
problem against the oracle.
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


def usable_context_check(ml, oracle_mod):
    prob = W.small_coupled(seed=0, shape=(37, 22, 29))
    g = ml.Grid(prob, 0)
    o = oracle_mod.OracleSim(prob)
    try:
        g.step(20)
        o.step(20)
        g.sync()
        for a, b in zip(g.fields(), o.fields()):
            assert rel(a, b) < 1e-4
    finally:
        g.close()


@pytest.mark.parametrize("shape", [(40, 24, 30), (96, 40, 36)])
def test_wait_timeout_reported(ml, oracle_mod, shape):
    prob = W.small_coupled(seed=1, shape=shape)
    g = ml.Grid(prob, 0)
    try:
        g.step(3)
        assert ml.ml_sync_status_code(g.h, g.stream) == ml.ML_OK
        ml.ml_set_wait_limit(g.h, 0)
        g.step(1)
        assert ml.ml_sync_status_code(g.h, g.stream) == ml.ML_ERR_TIMEOUT
        # the status was cleared by the read; with the default bound the steps run again
        ml.ml_set_wait_limit(g.h, 2000)
        g.step(2)
        assert ml.ml_sync_status_code(g.h, g.stream) == ml.ML_OK
        with pytest.raises(ml.MaxlinkError) as e:
            ml.ml_set_wait_limit(g.h, -1)
        assert e.value.status == ml.ML_ERR_INVALID_ARG
    finally:
        g.close()
    usable_context_check(ml, oracle_mod)


def test_wait_timeout_in_a_batch(ml):
    probs = [W.small_coupled(seed=s, shape=(37 + s, 22, 29)) for s in range(3)]
    grids = [ml.Grid(p, 0) for p in probs]
    b = ml.Batch(grids)
    try:
        b.step(2)
        for g in grids:
            assert ml.ml_sync_status_code(g.h, 0) == ml.ML_OK
        ml.ml_set_wait_limit(grids[1].h, 0)
        b.step(1)
        codes = [ml.ml_sync_status_code(g.h, 0) for g in grids]
        assert codes[1] == ml.ML_ERR_TIMEOUT
        assert codes[0] == ml.ML_OK and codes[2] == ml.ML_OK
    finally:
        b.close()
        for g in grids:
            g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_field_reported(ml, oracle_mod, precision):
    mols = W.pack_molecules([W.tls((20.3, 17.8, 14.6), 0.25, 0.5, sigma=1.5, cg=np.sqrt(0.9), ce=np.sqrt(0.1))])
    prob = W.Problem(40, 36, 30, 0.5, pml=(6,) * 6, molecules=mols)
    g = ml.Grid(prob, precision)
    try:
        g.step(2)
        assert ml.ml_sync_status_code(g.h, g.stream) == ml.ML_OK
        f = g.fields()
        f[2][14, 17, 20] = np.nan  # Ez inside the molecule's kernel window
        g.set_fields(f)
        g.step(1)
        assert ml.ml_sync_status_code(g.h, g.stream) == ml.ML_ERR_NUMERIC
        assert ml.ml_sync_status_code(g.h, g.stream) == ml.ML_OK  # cleared by the read
        with pytest.raises(ml.MaxlinkError) as e:
            g.step(1)
            g.sync()
        assert e.value.status == ml.ML_ERR_NUMERIC
    finally:
        g.close()
    usable_context_check(ml, oracle_mod)
