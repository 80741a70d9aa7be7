"""GPU discrete adjoint (ml_adjoint_run) against the oracle's adjoint on the same
seeded problems: objective, d/d eps over the design box and d/d gamma per
molecule, for exact two-level emitters and RK4 GKSL systems of up to 8 levels.  FP64
runs agree to round-off; FP32 runs within 1e-4 relative L2 (gradients) and 1e-5
(objective): the measured FP32 errors on these problems are at most 9e-7 and 8e-8.  Also: the result does not depend on the checkpoint interval (up to the
round-off of the per-segment gradient sums), the grid ends in the state a plain run
reaches, and unsupported inputs (zero couplings, no design box) are refused.
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


def coupled(seed, shape=(14, 12, 20), periodic=(False, True, False), drude=False, nmol=3, pml=3, lorentz=False):
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    zc = nz // 2
    mats = [W.tls([rng.uniform(4, nx - 5), rng.uniform(4, ny - 5), rng.uniform(zc + 1, zc + 3)], 0.3, 0.8,
                  axis=q % 3, sigma=0.8, gamma=rng.uniform(0.5, 1.5), cg=np.sqrt(0.7), ce=np.sqrt(0.3))
            for q in range(nmol)]
    box = (0 if drude else 3, 2, zc - 4, min(nx - 4, 8), min(ny - 3, 6), 4)
    deps = 1.0 + rng.uniform(0, 1.5, (box[5], box[4], box[3]))
    kw = {}
    if drude:
        m = np.zeros((nz, ny, nx), np.uint8)
        m[zc + 4:zc + 7, 2:6, nx - 7:nx - 3] = 1
        media = [W.Material(), W.Material(eps_inf=1.2, wp=0.9, gamma=0.05)]
        if lorentz:
            # a Lorentz oscillator and a three-pole material next to the Drude block
            m[zc + 4:zc + 7, 6:10, nx - 7:nx - 3] = 2
            m[pml + 1:pml + 3, 2:ny - 2, 2:nx - 2] = 3
            media += [W.Material(eps_inf=1.5, wp=0.5, gamma=0.02, omega0=0.3),
                      W.Material(eps_inf=1.1, wp=0.4, gamma=0.03, omega0=0.35,
                                 extra=((0.3, 0.05, 0.5), (0.5, 0.08, 0.0)))]
        kw = dict(mat=m, materials=media)
    p6 = tuple(0 if periodic[a // 2] else pml for a in range(6))
    return W.Problem(nx, ny, nz, 0.5, periodic=periodic, pml=p6, design_box=box, design_eps=deps,
                     sources=[W.Source(2, pml + 1, 0, 1.0, 0.3, 6.0, 18.0)],
                     planes=[W.FluxPlane(2, nz - pml - 2, np.array([0.25, 0.3]))],
                     molecules=W.pack_molecules(mats) if nmol else W.empty_molecules(), **kw)


def compare(ml, oracle_mod, prob, steps, precision, tol_obj, tol_grad, ckpt=25, freq=1):
    o = oracle_mod.OracleSim(prob)
    obj_o, ge_o, gg_o = o.adjoint_run(steps, 0, freq)
    x0, y0, z0, sx, sy, sz = prob.design_box
    ge_o = ge_o[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx]
    g = ml.Grid(prob, precision)
    try:
        obj, ge, gg = g.adjoint(steps, 0, freq, ckpt_every=ckpt)
    finally:
        g.close()
    assert abs(obj - obj_o) <= tol_obj * abs(obj_o)
    assert rel(ge, ge_o) < tol_grad
    if prob.molecules.count:
        assert rel(gg, gg_o) < tol_grad
    return obj, ge, gg


@pytest.mark.parametrize("precision,tol_obj,tol_grad", [(1, 1e-10, 1e-8), (0, 1e-5, 1e-4)])
def test_coupled_design_box_and_molecules(ml, oracle_mod, precision, tol_obj, tol_grad):
    compare(ml, oracle_mod, coupled(5), 80, precision, tol_obj, tol_grad)


@pytest.mark.parametrize("precision,tol_obj,tol_grad", [(1, 1e-10, 1e-8), (0, 1e-5, 1e-4)])
def test_drude_walls_ragged(ml, oracle_mod, precision, tol_obj, tol_grad):
    prob = coupled(6, shape=(37, 21, 26), periodic=(False, False, False), drude=True, nmol=4)
    compare(ml, oracle_mod, prob, 70, precision, tol_obj, tol_grad, ckpt=16)


def test_periodic_fields_only(ml, oracle_mod):
    prob = coupled(7, shape=(33, 10, 24), periodic=(True, True, False), nmol=0)
    compare(ml, oracle_mod, prob, 60, 1, 1e-10, 1e-8, ckpt=60, freq=0)


def test_checkpoint_interval_and_end_state(ml):
    prob = coupled(8)
    res = []
    for ckpt in (7, 1000):
        g = ml.Grid(prob, 1)
        try:
            res.append(g.adjoint(45, 0, 1, ckpt_every=ckpt) + (g.fields(), g.nstep))
        finally:
            g.close()
    (o1, e1, m1, f1, n1), (o2, e2, m2, f2, n2) = res
    # the permittivity gradient is folded into FP64 once per segment: round-off only
    assert o1 == o2 and np.array_equal(m1, m2) and rel(e1, e2) < 1e-12
    g = ml.Grid(prob, 1)
    try:
        g.step(45)
        plain = g.fields()
    finally:
        g.close()
    assert n1 == 45
    for a, b in zip(f1, plain):
        assert np.array_equal(a, b)


def test_setters_move_the_objective_as_the_gradient_says(ml):
    prob = coupled(9)
    g = ml.Grid(prob, 1)
    try:
        blob = g.checkpoint()
        obj, ge, gg = g.adjoint(60, 0, 1)
        h = 1e-4
        d = np.random.default_rng(0).standard_normal(ge.shape)
        vals = []
        for sgn in (1, -1):
            g.restore(blob)
            g.set_design_eps(prob.design_eps + sgn * h * d)
            vals.append(g.adjoint(60, 0, 1)[0])
        g.set_design_eps(prob.design_eps)
        assert abs((vals[0] - vals[1]) / (2 * h) - np.sum(ge * d)) < 1e-6 * abs(np.sum(ge * d))
        dg = np.random.default_rng(1).standard_normal(gg.shape)
        vals = []
        for sgn in (1, -1):
            g.restore(blob)
            g.set_couplings(prob.molecules.gamma + sgn * h * dg)
            vals.append(g.adjoint(60, 0, 1)[0])
        assert abs((vals[0] - vals[1]) / (2 * h) - gg @ dg) < 1e-6 * abs(gg @ dg)
    finally:
        g.close()


def with_multilevel(prob, seed, levels=(3, 5, 8), nsub=(1, 2, 1)):
    """The problem with RK4 GKSL systems (ladder decay and dephasing) added next to its
    two-level emitters."""
    rng = np.random.default_rng(seed)
    mol = prob.molecules
    mats = [dict(n=int(mol.nlev[m]), pos=mol.pos[m], sigma=mol.sigma[m], gamma=mol.gamma[m],
                 H0=mol.matrix(mol.H0, m), mu=np.stack([mol.matrix(mol.mu[a], m) for a in range(3)]),
                 rho=mol.matrix(mol.rho0, m), decay=mol.decay[m], dephase=mol.dephase[m], kind=int(mol.kind[m]),
                 nsub=int(mol.nsub[m])) for m in range(mol.count)]
    zc = prob.nz // 2
    for n, ns in zip(levels, nsub):
        mu = np.stack([W.random_hermitian(rng, n, 0.4) for _ in range(3)])
        c = rng.normal(size=n) + 1j * rng.normal(size=n)
        c /= np.linalg.norm(c)
        E = np.concatenate([[0.0], np.cumsum(0.3 * (1 + 0.05 * rng.uniform(-1, 1, n - 1)))])
        mats.append(dict(n=n, pos=[rng.uniform(4, prob.nx - 5), rng.uniform(4, prob.ny - 5), rng.uniform(zc + 1, zc + 3)],
                         sigma=0.8, gamma=rng.uniform(0.5, 1.5), H0=np.diag(E).astype(complex), mu=mu,
                         rho=np.outer(c, c.conj()), decay=0.02, dephase=0.01, kind=W.KIND_RK4, nsub=ns))
    return prob.replace(molecules=W.pack_molecules(mats))


@pytest.mark.parametrize("precision,tol_obj,tol_grad", [(1, 1e-10, 1e-8), (0, 1e-5, 1e-4)])
def test_multilevel_molecules_against_oracle(ml, oracle_mod, precision, tol_obj, tol_grad):
    """The reverse sweep through RK4 GKSL molecules (3, 5 and 8 levels, decay,
    dephasing, two substeps for one of them) next to exact two-level ones."""
    compare(ml, oracle_mod, with_multilevel(coupled(11), 11), 80, precision, tol_obj, tol_grad)


@pytest.mark.parametrize("precision,tol_obj,tol_grad", [(1, 1e-10, 1e-8), (0, 1e-5, 1e-4)])
def test_lorentz_and_multipole_media_against_oracle(ml, oracle_mod, precision, tol_obj, tol_grad):
    """The reverse sweep through Drude, Lorentz and three-pole cells (each slot's current
    and, for Lorentz poles, polarisation adjoint)."""
    prob = coupled(12, shape=(37, 21, 26), periodic=(False, False, False), drude=True, nmol=4, lorentz=True)
    compare(ml, oracle_mod, prob, 70, precision, tol_obj, tol_grad, ckpt=16)


_FULL = {}


@pytest.mark.parametrize("precision,tol_obj,tol_grad", [(1, 1e-10, 1e-8), (0, 1e-5, 1e-4)])
def test_design_problem_with_multilevel_molecules_and_media(ml, oracle_mod, precision, tol_obj, tol_grad):
    """A 64^3 copy of the inverse-design problem with every part of the step the adjoint
    takes at once: CPML on all faces, the design box, a source sheet, RK4 GKSL systems of
    2..8 levels, a Lorentz layer and a Drude + Lorentz film between the box and the flux
    plane."""
    prob = W.adjoint_design(n=64, design=12, nmol=12, pml=6, width=6.0, multilevel=True, media=True)
    if "o" not in _FULL:
        o = oracle_mod.OracleSim(prob)
        _FULL["o"] = o.adjoint_run(160, 0, 0)
    obj_o, ge_o, gg_o = _FULL["o"]
    x0, y0, z0, sx, sy, sz = prob.design_box
    g = ml.Grid(prob, precision)
    try:
        obj, ge, gg = g.adjoint(160, 0, 0, ckpt_every=40)
    finally:
        g.close()
    assert abs(obj - obj_o) <= tol_obj * abs(obj_o)
    assert rel(ge, ge_o[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx]) < tol_grad
    assert rel(gg, gg_o) < tol_grad


def test_refuses_unsupported_inputs(ml):
    mol = W.pack_molecules([W.tls([7.0, 6.0, 10.0], 0.3, 0.5, sigma=1.0, gamma=0.0, decay=0.01)])
    prob = W.Problem(14, 12, 20, 0.5, molecules=mol, planes=[W.FluxPlane(2, 15, np.array([0.3]))])
    g = ml.Grid(prob, 0)
    try:
        with pytest.raises(ml.MaxlinkError) as e:
            g.adjoint(5, 0, 0)
        assert e.value.status == ml.ML_ERR_INVALID_ARG
        buf = np.zeros(16)
        with pytest.raises(ml.MaxlinkError):
            ml.ml_adjoint_run(g.h, 5, 10, 0, 0, grad_eps_ptr=buf.ctypes.data)  # no design box
    finally:
        g.close()


def design_copy():
    """24^3 copy of the inverse-design workload (design box, emitters, pulse, far plane)."""
    return W.adjoint_design(n=24, design=10, nmol=20, pml=4, sigma=1.0, width=6.0, mol_x=(8.0, 11.0), seed=14)


@pytest.mark.parametrize("precision,tol_obj,tol_grad", [(1, 1e-10, 1e-8), (0, 1e-5, 1e-4)])
def test_design_workload_copy_matches_oracle(ml, oracle_mod, precision, tol_obj, tol_grad):
    compare(ml, oracle_mod, design_copy(), 150, precision, tol_obj, tol_grad, ckpt=40, freq=0)


def test_autograd_function(ml):
    import torch
    from paper_2512_06173_gb300.autograd import CoupledFlux
    prob = design_copy()
    g = ml.Grid(prob, 1)
    try:
        state0 = g.checkpoint()
        obj_ref, ge_ref, gg_ref = g.adjoint(150, 0, 0, ckpt_every=40)
        eps = torch.tensor(prob.design_eps, dtype=torch.float64, device="cuda", requires_grad=True)
        gam = torch.tensor(prob.molecules.gamma, dtype=torch.float64, device="cuda", requires_grad=True)
        J = CoupledFlux.apply(eps, gam, g, state0, 150, 0, 0, 40)
        assert abs(J.item() - obj_ref) <= 1e-12 * abs(obj_ref)
        # no input needs a gradient: the forward steps alone give the same objective
        J0 = CoupledFlux.apply(eps.detach(), gam.detach(), g, state0, 150, 0, 0, 40)
        assert not J0.requires_grad and abs(J0.item() - obj_ref) <= 1e-12 * abs(obj_ref)
        (2.0 * J).backward()
        np.testing.assert_allclose(eps.grad.cpu().numpy(), 2.0 * ge_ref, rtol=1e-12, atol=0)
        np.testing.assert_allclose(gam.grad.cpu().numpy(), 2.0 * gg_ref, rtol=1e-12, atol=0)
        # one small ascent step on eps raises the transmitted flux
        with torch.no_grad():
            step = 1e-2 / eps.grad.abs().max()
            eps2 = (eps + step * eps.grad).clamp_min(1.0)
        J2 = CoupledFlux.apply(eps2, gam.detach(), g, state0, 150, 0, 0, 40)
        assert J2.item() > J.item()
    finally:
        g.close()


@pytest.mark.slow
def test_full_size_gradient_entries_against_central_differences(ml):
    """192^3 inverse-design workload, FP64, 3000 steps: 10 design-box permittivities
    and 10 couplings against central differences with h = 1e-3."""
    prob = W.adjoint_design()
    g = ml.Grid(prob, 1)
    try:
        state0 = g.checkpoint()
        obj, ge, gg = g.adjoint(3000, 0, 0, ckpt_every=100)
        rng = np.random.default_rng(0)
        h = 1e-3
        cells = [tuple(rng.integers(0, 96, 3)) for _ in range(10)]
        mols = rng.choice(prob.molecules.count, 10, replace=False)

        def J():  # state0 has empty DFT sums, so a plain run gives the same objective
            g.step(3000)
            return g.flux(0)[0]

        scale_e = np.abs(ge).max()
        for c in cells:
            vals = []
            for sgn in (1, -1):
                e = prob.design_eps.copy()
                e[c] += sgn * h
                g.restore(state0)
                g.set_design_eps(e)
                vals.append(J())
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - ge[c]) <= 1e-3 * abs(ge[c]) + 1e-6 * scale_e
        g.set_design_eps(prob.design_eps)
        scale_g = np.abs(gg).max()
        for m in mols:
            vals = []
            for sgn in (1, -1):
                gm = prob.molecules.gamma.copy()
                gm[m] += sgn * h
                g.restore(state0)
                g.set_couplings(gm)
                vals.append(J())
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - gg[m]) <= 1e-3 * abs(gg[m]) + 1e-6 * scale_g
    finally:
        g.close()
