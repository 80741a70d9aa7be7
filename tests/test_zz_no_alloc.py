"""ml_gather_static, the allocation-free gather, against the gather inside a grid's
step on the same field.

The entry point serves callers that cannot let a library allocate device memory
(their memory is reserved by their own allocator, or an allocation's possible
device synchronisation is not acceptable where they call it).  Its scratch is a
fixed array inside the library; these tests check that two calls in a row both
reproduce the regularised field that ml_step computes, that counts beyond the
scratch's limit are refused, and that an empty call does nothing.  The file is
named to be collected last, so that it also runs after every other GPU test has
used the device.
"""
import math

import numpy as np
import pytest

from paper_2512_06173_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL32 = 1e-4  # relative L2, FP32 sums in a different order on each side


@pytest.fixture(scope="module")
def ml():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2512_06173_gb300 import maxlink
    maxlink.load()
    return maxlink


def ensemble(seed, shape, periodic, nmol):
    """Two-level molecules with dipoles along all three axes (so the grid gathers
    every component), random widths up to the largest window, windows inside the
    grid on wall axes and anywhere (wrapping) on periodic ones."""
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(nmol):
        sigma = rng.uniform(0.4, 7.0 / 3.0)
        R = math.ceil(3.0 * sigma)
        pos = []
        for ax, n in enumerate(shape):
            pos.append(rng.uniform(0.0, n) if periodic[ax] else rng.uniform(R, n - R - 1.0 - 1e-6))
        d = rng.standard_normal(3)
        mu = np.zeros((3, 2, 2), np.complex128)
        for ax in range(3):
            mu[ax] = d[ax] * np.array([[0, 1], [1, 0]])
        mats.append(dict(n=2, pos=pos, sigma=sigma, gamma=rng.uniform(0.5, 2.0),
                         H0=np.diag([0.0, 0.3]), mu=mu, rho=np.diag([1.0, 0.0])))
    return W.pack_molecules(mats)


CASES = [
    # (nx, ny, nz), periodic flags, molecules
    ((45, 26, 33), (True, False, True), 40),
    ((38, 20, 9), (False, True, True), 25),   # z shorter than the widest window: it folds
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_matches_grid_gather_twice(ml, case):
    import torch
    (nx, ny, nz), periodic, nmol = CASES[case]
    mol = ensemble(10 + case, (nx, ny, nz), periodic, nmol)
    prob = W.Problem(nx, ny, nz, 0.5, periodic=periodic, molecules=mol)
    g = ml.Grid(prob, ml.ML_F32)
    try:
        g.set_fields(W.random_fields(prob, 20 + case))
        N = nx * ny * nz
        E = torch.empty(3 * N, dtype=torch.float32, device="cuda")
        ml.ml_get_fields(g.h, ml.ML_EX | ml.ML_EY | ml.ML_EZ, E.data_ptr(), True, 0)
        g.step(1)  # the step gathers from the field it starts with
        g.sync()
        want = g.molecules(ml.ML_MOL_EFIELD)
    finally:
        g.close()
    assert np.all(np.abs(want) > 0)

    pos = torch.tensor(mol.pos, dtype=torch.float64, device="cuda")
    sigma = torch.tensor(mol.sigma, dtype=torch.float64, device="cuda")
    gamma = torch.tensor(mol.gamma, dtype=torch.float64, device="cuda")
    out = torch.empty((nmol, 3), dtype=torch.float32, device="cuda")
    scale = float(np.abs(want).max())
    for _ in range(2):
        out.fill_(float("nan"))
        ml.ml_gather_static(E.data_ptr(), nx, ny, nz, periodic, nmol, pos.data_ptr(), sigma.data_ptr(),
                            gamma.data_ptr(), out.data_ptr(), 0)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < TOL32
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-4 * scale)


def test_limits(ml):
    import torch
    E = torch.zeros(3 * 8, dtype=torch.float32, device="cuda")
    with pytest.raises(ml.MaxlinkError) as e:
        ml.ml_gather_static(E.data_ptr(), 2, 2, 2, (0, 0, 0), ml.ML_STATIC_GATHER_MAX_MOLECULES + 1,
                            E.data_ptr(), E.data_ptr(), E.data_ptr(), E.data_ptr(), 0)
    assert e.value.status == ml.ML_ERR_INVALID_ARG
    assert str(ml.ML_STATIC_GATHER_MAX_MOLECULES) in str(e.value)
    # nothing to do: returns without touching any pointer
    ml.ml_gather_static(E.data_ptr(), 2, 2, 2, (0, 0, 0), 0, 0, 0, 0, 0, 0)
    torch.cuda.synchronize()
