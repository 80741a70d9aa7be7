"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs, element by element.

Tolerances: FP64 GPU runs agree with the oracle to round-off (relative L2 <= 1e-10;
the summation order of the molecular current and the kernel sums differ); FP32
runs agree within relative L2 <= 1e-4 for fields, density matrices, excited-level
populations, dipole rates d<mu>/dt, regularised fields, energy sums and flux spectra
(measured FP32 errors are 1e-8 .. 1e-5).
"""
import numpy as np
import pytest

from paper_2512_06173_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-4


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
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def crel(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def excited(pops, prob):
    """Populations of the excited levels (1 .. n-1) of every molecule, concatenated."""
    nl = prob.molecules.nlev
    return np.concatenate([pops[m, 1:int(nl[m])] for m in range(prob.molecules.count)])


def run_pair(ml, oracle_mod, prob, steps, precision, fields=None, molecules=True):
    g = ml.Grid(prob, precision, molecules=molecules)
    o = oracle_mod.OracleSim(prob, molecules=molecules)
    if fields is not None:
        g.set_fields(fields)
        o.set_fields(fields)
    g.step(steps)
    o.step(steps)
    g.sync()
    return g, o


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
@pytest.mark.parametrize("shape", [(37, 21, 19), (64, 16, 9), (5, 3, 40)])
def test_vacuum_cpml_fields(ml, oracle_mod, precision, tol, shape):
    nx, ny, nz = shape
    pml = tuple(min(4, n // 3) for n in (nx, nx, ny, ny, nz, nz))
    prob = W.Problem(nx, ny, nz, 0.5, pml=pml)
    f = W.random_fields(prob, 5)
    g, o = run_pair(ml, oracle_mod, prob, 30, precision, fields=f)
    for got, want in zip(g.fields(), o.fields()):
        assert rel(got, want) < tol


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
@pytest.mark.parametrize("per", [(True, True, True), (True, False, True), (False, True, False)])
@pytest.mark.parametrize("shape", [(33, 10, 12), (64, 24, 12)])  # nx % 8 == 0: sector-wide x images
def test_periodic_and_walls(ml, oracle_mod, precision, tol, per, shape):
    nx, ny, nz = shape
    pml = tuple(0 if per[a // 2] else 3 for a in range(6))
    prob = W.Problem(nx, ny, nz, 0.5, periodic=per, pml=pml)
    f = W.random_fields(prob, 8)
    g, o = run_pair(ml, oracle_mod, prob, 25, precision, fields=f)
    for got, want in zip(g.fields(), o.fields()):
        assert rel(got, want) < tol


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
def test_thin_periodic_layer(ml, oracle_mod, precision, tol):
    """nz = 1 periodic: the 2D limit used by the paper's superradiance example."""
    mols = W.pack_molecules([W.tls((20.3, 17.8, 0.4), 0.25, 0.5, sigma=1.0, cg=np.sqrt(0.99), ce=0.1),
                             W.tls((11.0, 25.5, 0.9), 0.3, 0.4, sigma=1.5, cg=np.sqrt(0.5), ce=np.sqrt(0.5))])
    prob = W.Problem(40, 36, 1, 0.5, periodic=(False, False, True), pml=(6, 6, 6, 6, 0, 0), molecules=mols)
    g, o = run_pair(ml, oracle_mod, prob, 120, precision)
    for got, want in zip(g.fields(), o.fields()):
        assert rel(got, want) < tol
    assert crel(np.concatenate([g.rho(m).ravel() for m in range(2)]),
                np.concatenate([o.rho(m).ravel() for m in range(2)])) < tol


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
def test_printed_superradiance_example(ml, oracle_mod, precision, tol):
    """The paper's printed superradiance example (Appendix B, tests/golden): four
    co-located two-level systems at a coupling of 1.0 in grid units, a one-cell kernel,
    an 80 x 80 cell with 30-cell absorbing layers, nz = 1 periodic; 200 steps (the
    excited population falls to about a quarter).  Coherences, populations and fields."""
    import json
    from test_oracle_golden import GOLDEN, grid_units
    gd = json.load(open(GOLDEN))
    _, n, pml, w, mu = grid_units(gd)
    cg, ce = np.sqrt(gd["initial_state"]["cg_squared"]), gd["initial_state"]["ce"]
    mols = W.pack_molecules([W.tls((n / 2, n / 2, 0.5), w, mu, axis=2, sigma=1.0, gamma=1.0, cg=cg, ce=ce)
                             for _ in range(4)])
    prob = W.Problem(n, n, 1, 0.5, periodic=(False, False, True), pml=(pml, pml, pml, pml, 0, 0), molecules=mols)
    g, o = run_pair(ml, oracle_mod, prob, 200, precision)
    try:
        for got, want in zip(g.fields(), o.fields()):
            assert rel(got, want) < tol
        r_g = [g.rho(m) for m in range(4)]
        r_o = [o.rho(m) for m in range(4)]
        assert crel(np.array([r[0, 1] for r in r_g]), np.array([r[0, 1] for r in r_o])) < tol
        pe_o = np.array([r[1, 1].real for r in r_o])
        assert pe_o.max() < 0.5e-4  # decayed from 1e-4
        assert rel([r[1, 1].real for r in r_g], pe_o) < tol
    finally:
        g.close()


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_coupled_all_features(ml, oracle_mod, precision, tol, seed):
    """eps map + design box + source sheet + flux planes + two-level and multilevel
    Lindblad molecules on a ragged grid."""
    prob = W.small_coupled(seed=seed, shape=(37 + seed, 22, 29))
    g, o = run_pair(ml, oracle_mod, prob, 60, precision)
    for got, want in zip(g.fields(), o.fields()):
        assert rel(got, want) < tol
    M = prob.molecules.count
    assert crel(np.concatenate([g.rho(m).ravel() for m in range(M)]),
                np.concatenate([o.rho(m).ravel() for m in range(M)])) < tol
    pops = g.molecules(ml.ML_MOL_POP)
    assert rel(excited(pops, prob), np.concatenate([np.real(np.diag(o.rho(m)))[1:] for m in range(M)])) < tol
    # the enqueued readback into page-locked memory gives the same bytes once the
    # stream has reached it
    import torch
    pinned = torch.zeros(pops.size, dtype=torch.float64).pin_memory()
    ml.ml_get_molecules(g.h, ml.ML_MOL_POP, pinned.data_ptr(), ml.ML_HOST_ASYNC, g.stream)
    torch.cuda.synchronize()
    assert np.array_equal(pinned.numpy().reshape(pops.shape), pops)
    md = g.molecules(ml.ML_MOL_MUDOT)
    assert rel(md, np.array([o.mol_state(m)[1] for m in range(M)])) < tol
    for p in range(len(prob.planes)):
        fg, fo = g.flux(p), o.flux(p)
        assert rel(fg, fo) < (1e-9 if precision == 1 else tol)


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
def test_bragg_resonator_copy(ml, oracle_mod, precision, tol):
    """Small copy of the Bragg-resonator ensemble: layer stack along x, multilevel
    Lindblad systems (2..8 levels) in the central slab, z-polarised pulse sheet, flux
    planes on both sides; 120 steps so that the pulse reaches the slab."""
    prob = W.bragg_ensemble(nx=96, ny=40, nz=36, nmol=30, pml=4, slab=8, layers=4, width=6.0)
    g, o = run_pair(ml, oracle_mod, prob, 120, precision)
    # the field is z-polarised: components that stay near zero are measured against
    # the largest component's norm
    fo = o.fields()
    scale = max(np.linalg.norm(f) for f in fo)
    for got, want in zip(g.fields(), fo):
        assert np.linalg.norm(np.asarray(got, np.float64) - want) < tol * scale
    M = prob.molecules.count
    pops = g.molecules(ml.ML_MOL_POP)
    assert rel(excited(pops, prob), np.concatenate([np.real(np.diag(o.rho(m)))[1:] for m in range(M)])) < tol
    assert rel(g.molecules(ml.ML_MOL_MUDOT), np.array([o.mol_state(m)[1] for m in range(M)])) < tol
    # the far plane has not seen the pulse yet: errors against the larger flux
    fl = [(g.flux(p), o.flux(p)) for p in range(len(prob.planes))]
    fscale = max(np.abs(fo).max() for _, fo in fl)
    for fg, fo in fl:
        assert np.abs(fg - fo).max() < (1e-9 if precision == 1 else tol) * fscale


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
def test_drude_sphere(ml, oracle_mod, precision, tol):
    prob = W.small_coupled(seed=4, shape=(30, 30, 30), drude=True, eps_map=False, nmol=4, planes=False)
    g, o = run_pair(ml, oracle_mod, prob, 80, precision)
    for got, want in zip(g.fields(), o.fields()):
        assert rel(got, want) < tol
    ab_g, ab_o = g.absorbed(), o.absorbed()
    assert abs(ab_g - ab_o) <= (1e-9 if precision == 1 else tol) * abs(ab_o)


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
def test_lorentz_drude_sphere(ml, oracle_mod, precision, tol):
    """One pole box holding a Drude half-sphere and a Lorentz half-sphere (the restoring
    term and the polarisation update of the pole ADE), with molecules and a source."""
    prob = W.small_coupled(seed=7, shape=(30, 28, 33), drude=True, lorentz=True, eps_map=False, nmol=4,
                           planes=False)
    g, o = run_pair(ml, oracle_mod, prob, 160, precision)
    for got, want in zip(g.fields(), o.fields()):
        assert rel(got, want) < tol
    ab_g, ab_o = g.absorbed(), o.absorbed()
    assert abs(ab_g - ab_o) <= (1e-9 if precision == 1 else tol) * abs(ab_o)
    M = prob.molecules.count
    pops = g.molecules(ml.ML_MOL_POP)
    assert rel(excited(pops, prob), np.concatenate([np.real(np.diag(o.rho(m)))[1:] for m in range(M)])) < tol


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
def test_dispersive_stack_small(ml, oracle_mod, precision, tol):
    """The dispersive-stack workload's generator at 26x22x64 (periodic x and y, ragged
    tiles): a pulse through the Lorentz layer onto the Drude film, emitters in the
    layer, flux on both sides, 220 steps."""
    prob = W.dispersive_stack(nx=26, ny=22, nz=64, nmol=7, pml=6, layer=16, film=4, width=6.0, t0=18.0)
    g, o = run_pair(ml, oracle_mod, prob, 220, precision)
    fo = o.fields()
    scale = max(np.linalg.norm(f) for f in fo)
    for got, want in zip(g.fields(), fo):
        assert np.linalg.norm(np.asarray(got, np.float64) - want) < tol * scale
    pops = g.molecules(ml.ML_MOL_POP)
    pe_o = np.array([np.real(o.rho(m)[1, 1]) for m in range(prob.molecules.count)])
    assert pe_o.max() > 1e-6  # the pulse has reached the emitters
    assert rel(pops[:, 1], pe_o) < tol
    for p in range(len(prob.planes)):
        fg, fw = g.flux(p), o.flux(p)
        assert np.abs(fg - fw).max() < (1e-9 if precision == 1 else tol) * np.abs(fw).max()
    ab_g, ab_o = g.absorbed(), o.absorbed()
    assert abs(ab_g - ab_o) <= (1e-9 if precision == 1 else tol) * abs(ab_o)


def test_lorentz_checkpoint(ml):
    """The polarisation is part of the saved state."""
    prob = W.small_coupled(seed=8, shape=(26, 24, 28), drude=True, lorentz=True, nmol=3)
    g = ml.Grid(prob, 1)
    g.step(30)
    blob = g.checkpoint()
    g.step(50)
    a = g.fields()
    g.restore(blob)
    g.step(50)
    for x, y in zip(a, g.fields()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, 1e-4)])
def test_plain_single_emitter_trajectory(ml, oracle_mod, precision, tol):
    """40^3 cells, one emitter at the centre, 1000 steps; excited population every
    step and Ez along the centre line."""
    prob = W.plain_single_emitter()
    g = ml.Grid(prob, precision)
    o = oracle_mod.OracleSim(prob)
    pe_g, pe_o = [], []
    for _ in range(1000):
        g.step(1)
        o.step(1)
        pe_g.append(g.molecules(ml.ML_MOL_POP)[0, 1])
        pe_o.append(o.rho(0)[1, 1].real)
    assert rel(pe_g, pe_o) < tol
    ez_g = g.fields(ml.ML_EZ)[0][:, 20, 20]
    ez_o = o.fields()[2][:, 20, 20]
    assert rel(ez_g, ez_o) < tol


def test_checkpoint_roundtrip(ml):
    prob = W.small_coupled(seed=5, shape=(24, 20, 22))
    g = ml.Grid(prob, 0)
    g.step(17)
    blob = g.checkpoint()
    g.step(23)
    a = g.fields()
    ra = g.molecules(ml.ML_MOL_RHO)
    fa = g.flux(0)
    g.restore(blob)
    assert g.nstep == 17
    g.step(23)
    b = g.fields()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.array_equal(ra, g.molecules(ml.ML_MOL_RHO))
    assert np.array_equal(fa, g.flux(0))


def test_deterministic_repeat(ml):
    prob = W.small_coupled(seed=6, shape=(40, 24, 30))
    outs = []
    for _ in range(2):
        g = ml.Grid(prob, 0)
        g.step(40)
        outs.append((g.fields(), g.molecules(ml.ML_MOL_RHO)))
    for x, y in zip(outs[0][0], outs[1][0]):
        assert np.array_equal(x, y)
    assert np.array_equal(outs[0][1], outs[1][1])


def test_window_crossing_wall_rejected(ml):
    mols = W.pack_molecules([W.tls((1.5, 8.0, 8.0), 0.25, 0.1, sigma=1.5)])
    prob = W.Problem(16, 16, 16, 0.5, molecules=mols)
    with pytest.raises(ml.MaxlinkError) as e:
        ml.Grid(prob, 0)
    assert e.value.status == ml.ML_ERR_INVALID_ARG


@pytest.mark.parametrize("two_level", [False, True])
def test_population_sink(ml, two_level):
    """The molecule kernel's stores into the page-locked ring equal the populations read
    back after each step (bit for bit), in the slot of that step; entries past a
    molecule's levels and slots of other steps are left alone."""
    import torch
    prob = (W.superradiant_slab(n=48, nmol=40, slab=8, pml=6) if two_level
            else W.small_coupled(seed=4, shape=(37, 22, 29)))
    M, L, ring = prob.molecules.count, ml.ML_MAX_LEVELS, 3
    g = ml.Grid(prob, 0)
    try:
        sink = torch.full((ring * M * L,), -7.0, dtype=torch.float64).pin_memory()
        ml.ml_set_population_sink(g.h, sink.data_ptr(), ring)
        nlev = prob.molecules.nlev
        for s in range(5):
            g.step(1)
            g.sync()
            want = g.molecules(ml.ML_MOL_POP)
            got = sink.numpy().reshape(ring, M, L)[s % ring]
            for m in range(M):
                assert np.array_equal(got[m, :nlev[m]], want[m, :nlev[m]])
                assert np.all(got[m, nlev[m]:] == -7.0)
        ml.ml_set_population_sink(g.h, 0, 1)
        before = sink.clone()
        g.step(2)
        g.sync()
        assert torch.equal(sink, before)
        with pytest.raises(ml.MaxlinkError):
            ml.ml_set_population_sink(g.h, sink.data_ptr(), 0)
    finally:
        g.close()


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
@pytest.mark.parametrize("seed", [0, 3])
def test_molecule_field_and_energy(ml, oracle_mod, precision, tol, seed):
    """The regularised field of the last step (Eq. E_regu_Emi, ML_MOL_EFIELD) and the
    FP64 running sum of Tr(rho H0) over the steps (ML_MOL_ENERGY) of every molecule,
    two-level and multilevel, against the oracle's."""
    prob = W.small_coupled(seed=seed, shape=(37, 22, 29))
    g, o = run_pair(ml, oracle_mod, prob, 60, precision)
    mol = prob.molecules
    M = mol.count
    st = [o.mol_state(m) for m in range(M)]
    et_o = np.array([s[0] for s in st])
    en_o = np.array([s[2] for s in st])
    # the components along which a molecule has a dipole (the others do not enter its
    # Hamiltonian and are not gathered: they read 0)
    cm = np.array([[np.any(mol.matrix(mol.mu[c], m) != 0) for c in range(3)] for m in range(M)])
    et_g = g.molecules(ml.ML_MOL_EFIELD)
    assert np.abs(et_o[cm]).max() > 0 and np.all(et_g[~cm] == 0)
    assert rel(et_g[cm], et_o[cm]) < tol
    assert rel(g.molecules(ml.ML_MOL_ENERGY), en_o) < tol


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
@pytest.mark.parametrize("case", ["material", "source"])
def test_material_and_source_bodies(ml, oracle_mod, precision, tol, case):
    """Grids large enough for tiles clear of every layer and wall: a layer stack across
    interior tiles (the material body of the field pass: dt/eps from the material table)
    and a source sheet crossing interior tiles and CPML tiles (the interior-geometry and
    CPML bodies with a source), with molecules, against the oracle."""
    if case == "material":
        prob = W.bragg_ensemble(nx=136, ny=40, nz=44, nmol=12, pml=4, slab=8, layers=6, width=6.0)
    else:
        prob = W.small_coupled(seed=3, shape=(70, 30, 40), eps_map=False, nmol=6)
    g, o = run_pair(ml, oracle_mod, prob, 120, precision)
    fo = o.fields()
    scale = max(np.linalg.norm(f) for f in fo)
    for got, want in zip(g.fields(), fo):
        assert np.linalg.norm(np.asarray(got, np.float64) - want) < tol * scale
    M = prob.molecules.count
    ro = [o.rho(m) for m in range(M)]
    assert crel(np.concatenate([g.rho(m).ravel() for m in range(M)]), np.concatenate([r.ravel() for r in ro])) < tol


@pytest.mark.parametrize("precision,tol", [(1, TOL64), (0, TOL32)])
def test_narrow_kernels(ml, oracle_mod, precision, tol):
    """Kernels far narrower than a cell (sigma = 0.01 and 0.005, where every sample's
    Gaussian underflows unless it is taken relative to the nearest sample): finite
    regularised fields and currents equal to the oracle's."""
    mols = W.pack_molecules([W.tls((6.5, 5.5, 7.5), 0.25, 0.5, axis=a, sigma=sg, cg=np.sqrt(0.7), ce=np.sqrt(0.3))
                             for a, sg in ((0, 0.01), (2, 0.005), (1, 0.01))])
    mols.pos[2] = (9.0, 6.0, 5.0)
    prob = W.Problem(16, 13, 14, 0.5, pml=(3,) * 6, molecules=mols)
    f = W.random_fields(prob, 4)
    g, o = run_pair(ml, oracle_mod, prob, 5, precision, fields=f)
    et = g.molecules(ml.ML_MOL_EFIELD)
    et_o = np.array([o.mol_state(m)[0] for m in range(3)])
    cm = np.array([[a == b for b in range(3)] for a in (0, 2, 1)])
    assert np.all(np.isfinite(et)) and np.all(np.isfinite(g.molecules(ml.ML_MOL_MUDOT)))
    assert rel(et[cm], et_o[cm]) < tol
    for got, want in zip(g.fields(), o.fields()):
        assert rel(got, want) < tol

