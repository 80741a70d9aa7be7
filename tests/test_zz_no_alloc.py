"""ml_gather_static, the allocation-free gather, against the gather inside a grid's
step on the same field, against the oracle's gather, and against Eq. E_regu_Emi
restated here with numpy (for windows that cross a wall, which the oracle's grid
refuses).

The entry point serves callers that cannot let a library allocate device memory
(their memory is reserved by their own allocator, or an allocation's possible
device synchronisation is not acceptable where they call it).  Its scratch is a
fixed array inside the library; these tests check that two calls in a row both
reproduce the regularised field that ml_step computes, that windows crossing a wall
leave the outside cells out of the sum, that kernels far narrower than a cell give
the mean of the nearest samples, that invalid widths give NaN, that counts beyond the
scratch's limit are refused, and that an empty call does nothing.  The file is named
to be collected last, so that it also runs after every other GPU test has used the
device.
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
def test_matches_grid_gather_twice(ml, oracle_mod, case):
    import torch
    (nx, ny, nz), periodic, nmol = CASES[case]
    mol = ensemble(10 + case, (nx, ny, nz), periodic, nmol)
    prob = W.Problem(nx, ny, nz, 0.5, periodic=periodic, molecules=mol)
    fields = [f.astype(np.float32).astype(np.float64) for f in W.random_fields(prob, 20 + case)]
    # the oracle's gather (Eq. E_regu_Emi, FP64) of the same FP32 field
    o = oracle_mod.OracleSim(prob)
    o.set_fields(fields)
    want_o = np.array([o.gather(m) for m in range(nmol)])
    g = ml.Grid(prob, ml.ML_F32)
    try:
        g.set_fields(fields)
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
        assert np.linalg.norm(got - want_o) / np.linalg.norm(want_o) < TOL32


def restated_gather(E, pos, sigma, gamma, periodic):
    """Eq. E_regu_Emi written out with numpy: per axis the 2R+2 samples from floor(p)-R
    (R = ceil(3 sigma)), component c sampled half a cell along c, Gaussian weights
    normalised over the whole window; on a periodic axis indices wrap, on a wall axis
    cells outside the grid are left out of the sum (the weights are not renormalised)."""
    nz, ny, nx = E[0].shape
    dims = (nx, ny, nz)
    out = np.zeros((len(pos), 3))
    for m, (p, sg, gm) in enumerate(zip(pos, sigma, gamma)):
        R = math.ceil(3 * sg)
        for c in range(3):
            idx, wts = [], []
            for ax in range(3):
                s0 = math.floor(p[ax]) - R
                t = np.arange(s0, s0 + 2 * R + 2)
                d = t + (0.5 if ax == c else 0.0) - p[ax]
                w = np.exp(-(d * d - np.min(d * d)) / (2 * sg * sg))
                w /= w.sum()
                if periodic[ax]:
                    t = t % dims[ax]
                else:
                    keep = (t >= 0) & (t < dims[ax])
                    t, w = t[keep], w[keep]
                idx.append(t)
                wts.append(w)
            sub = E[c][np.ix_(idx[2], idx[1], idx[0])]
            out[m, c] = gm * np.einsum("k,j,i,kji->", wts[2], wts[1], wts[0], sub)
    return out


def test_walls_narrow_kernels_and_invalid_widths(ml):
    """Against the restated Eq. E_regu_Emi: windows that cross a wall (cells outside the
    grid left out), windows that wrap a periodic axis, kernels far narrower than a cell
    (sigma = 0.01 at a cell centre: the mean of the nearest samples), and widths outside
    (0, 7/3], which give NaN."""
    import torch
    nx, ny, nz = 30, 22, 26
    periodic = (False, True, False)
    rng = np.random.default_rng(7)
    E = [rng.standard_normal((nz, ny, nx)).astype(np.float32) for _ in range(3)]
    pos = [(0.7, 5.2, 13.1),       # crosses the x = 0 wall
           (28.6, 21.3, 24.9),     # crosses the x = nx and z = nz walls, wraps in y
           (14.5, 10.5, 12.5),     # narrow kernel at a cell centre
           (15.3, 0.2, 1.4),       # wraps y, crosses the z = 0 wall
           (12.0, 9.0, 9.0),       # sigma beyond 7/3: NaN
           (10.2, 8.8, 7.7)]       # sigma <= 0: NaN
    sigma = [1.5, 2.2, 0.01, 0.9, 2.5, 0.0]
    gamma = [1.1, 0.7, 1.3, 2.0, 1.0, 1.0]
    Ed = torch.tensor(np.concatenate([x.ravel() for x in E]), device="cuda")
    pd = torch.tensor(np.array(pos), dtype=torch.float64, device="cuda")
    sd = torch.tensor(sigma, dtype=torch.float64, device="cuda")
    gd = torch.tensor(gamma, dtype=torch.float64, device="cuda")
    out = torch.empty((len(pos), 3), dtype=torch.float32, device="cuda")
    ml.ml_gather_static(Ed.data_ptr(), nx, ny, nz, periodic, len(pos), pd.data_ptr(), sd.data_ptr(),
                        gd.data_ptr(), out.data_ptr(), 0)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    want = restated_gather([x.astype(np.float64) for x in E], pos[:4], sigma[:4], gamma[:4], periodic)
    assert np.all(np.isfinite(got[:4]))
    assert np.linalg.norm(got[:4] - want) / np.linalg.norm(want) < TOL32
    i, j, k = 14, 10, 12
    Ex = E[0].astype(np.float64)
    assert abs(got[2, 0] - 1.3 * 0.25 * (Ex[k, j, i] + Ex[k, j + 1, i] + Ex[k + 1, j, i] + Ex[k + 1, j + 1, i])) < 1e-5
    assert np.all(np.isnan(got[4:]))


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
