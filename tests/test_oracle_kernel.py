"""Pins of the oracle's Gaussian-kernel gather and scatter (Eq. Polarization_mol,
Eq. E_regu_Emi, Eq. J_mol).

Checked against: the normalisation |sum kappa dV| = 1 (uniform fields gather exactly
gamma * E); a brute-force non-separable 3D Gaussian written here with numpy; and the
exact duality sum_cells E . J dV = sum_m Etilde_m . mudot_m between gather and scatter.
"""
import numpy as np
import pytest

from paper_2512_06173_gb300.workloads import Problem, pack_molecules, random_fields, tls


def brute_gather(E, comp, pos, sigma, gamma, periodic):
    """Non-separable evaluation: 3D Gaussian at the component's staggered positions in
    the window of 2R+2 cells per axis starting at floor(pos)-R, normalised by its 3D sum."""
    nz, ny, nx = E.shape
    R = int(np.ceil(3 * sigma))
    starts = [int(np.floor(p)) - R for p in pos]
    rng_ = [np.arange(s, s + 2 * R + 2) for s in starts]
    II, JJ, KK = np.meshgrid(*rng_, indexing="ij")
    off = [0.0, 0.0, 0.0]
    off[comp] = 0.5
    d2 = (II + off[0] - pos[0]) ** 2 + (JJ + off[1] - pos[1]) ** 2 + (KK + off[2] - pos[2]) ** 2
    w = np.exp(-d2 / (2 * sigma ** 2))
    w /= w.sum()
    ii, jj, kk = II % nx, JJ % ny, KK % nz
    return gamma * (w * E[kk, jj, ii]).sum()


@pytest.mark.parametrize("periodic", [False, True])
def test_gather_bruteforce(oracle_mod, periodic):
    rng = np.random.Generator(np.random.PCG64(4))
    shape = (17, 15, 19)
    mols = []
    for q in range(5):
        sigma = [1.0, 1.5, 2.0, 0.7, 1.2][q]
        R = int(np.ceil(3 * sigma))
        if periodic:
            pos = tuple(rng.uniform(0, n) for n in (19, 15, 17))
        else:
            pos = tuple(rng.uniform(R + 1, n - R - 2) for n in (19, 15, 17))
        mols.append(tls(pos, 0.25, 0.1, sigma=sigma, gamma=float(rng.uniform(0.5, 2))))
    prob = Problem(19, 15, 17, 0.5, periodic=(periodic,) * 3, molecules=pack_molecules(mols))
    sim = oracle_mod.OracleSim(prob)
    f = random_fields(prob, 9)
    sim.set_fields(f)
    for m in range(5):
        got = sim.gather(m)
        for c in range(3):
            want = brute_gather(f[c], c, prob.molecules.pos[m], prob.molecules.sigma[m],
                                prob.molecules.gamma[m], periodic)
            assert abs(got[c] - want) < 1e-13 * max(1, abs(want))


def test_uniform_field_normalisation(oracle_mod):
    """kappa integrates to one for every component, including a window folded many
    times onto a single periodic layer (the 2D limit)."""
    mols = [tls((3.3, 4.1, 0.2), 0.25, 0.1, sigma=1.5, gamma=1.7),
            tls((0.1, 7.9, 0.9), 0.25, 0.1, sigma=2.0, gamma=0.6)]
    prob = Problem(8, 9, 1, 0.5, periodic=(True, True, True), molecules=pack_molecules(mols))
    sim = oracle_mod.OracleSim(prob)
    E0 = [0.3, -1.2, 2.5]
    sim.set_fields([np.full((1, 9, 8), e) for e in E0] + [np.zeros((1, 9, 8))] * 3)
    for m, g in enumerate([1.7, 0.6]):
        assert np.allclose(sim.gather(m), g * np.array(E0), rtol=1e-14, atol=0)


def test_gather_scatter_duality(oracle_mod, W):
    """Energy handed from the field to the molecules equals the work of the molecular
    current on the field: sum_cells E^n . J^{n+1/2} = sum_m Etilde_m^n . mudot_m."""
    prob = W.small_coupled(seed=3, eps_map=False, source=False, planes=False)
    sim = oracle_mod.OracleSim(prob)
    f = random_fields(prob, 21, scale=0.1)
    sim.set_fields(f)
    sim.step(1)
    J = sim.current()
    lhs = sum((f[c] * J[c]).sum() for c in range(3))
    rhs = 0.0
    for m in range(sim.nmol):
        Et, md, _ = sim.mol_state(m)
        rhs += float(np.dot(Et, md))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(rhs))
    assert abs(rhs) > 1e-6


def test_window_outside_wall_rejected(oracle_mod):
    mols = [tls((2.0, 8.0, 8.0), 0.25, 0.1, sigma=1.5)]
    prob = Problem(16, 16, 16, 0.5, molecules=pack_molecules(mols))
    sim = oracle_mod.OracleSim(prob)
    with pytest.raises(ValueError):
        sim.step(1)


@pytest.mark.parametrize("sigma", [0.01, 0.005])
def test_narrow_kernel_selects_the_nearest_samples(oracle_mod, sigma):
    """A kernel much narrower than a cell (Eq. Polarization_mol as sigma -> 0) weights only
    the samples nearest the centre, equally when two are equally near: for a molecule at
    a cell centre (i+1/2, j+1/2, k+1/2) the x component is sampled at x = i+1/2 exactly and
    at the two y and the two z samples half a cell away, so E~_x is gamma times the mean
    of four Ex values (and likewise for y, z).  exp(-d^2 / 2 sigma^2) underflows for
    every sample here; the normalised weights must still come out finite."""
    i, j, k = 6, 4, 5
    mols = [tls((i + 0.5, j + 0.5, k + 0.5), 0.25, 0.1, sigma=sigma, gamma=1.3)]
    prob = Problem(13, 11, 12, 0.5, molecules=pack_molecules(mols))
    sim = oracle_mod.OracleSim(prob)
    f = random_fields(prob, 31)
    sim.set_fields(f)
    Ex, Ey, Ez = f[0], f[1], f[2]
    want = 1.3 * 0.25 * np.array([
        Ex[k, j, i] + Ex[k, j + 1, i] + Ex[k + 1, j, i] + Ex[k + 1, j + 1, i],
        Ey[k, j, i] + Ey[k, j, i + 1] + Ey[k + 1, j, i] + Ey[k + 1, j, i + 1],
        Ez[k, j, i] + Ez[k, j, i + 1] + Ez[k, j + 1, i] + Ez[k, j + 1, i + 1]])
    got = sim.gather(0)
    assert np.all(np.isfinite(got))
    assert np.allclose(got, want, rtol=1e-13, atol=1e-15)
