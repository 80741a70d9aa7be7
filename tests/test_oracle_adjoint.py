"""Pins of the oracle's discrete adjoint (gradients of a DFT flux with respect to
per-cell permittivity and per-molecule coupling) against facts that do not come
from the adjoint code itself:

* dot-product identity <L x, y> = <x, L^T y> for the linear field step (CPML on
  some axes, periodic and wall axes, material table, Drude, Lorentz and three-pole
  cells): any dropped term, wrong sign or transposed index in the reversed step
  breaks it;
* the vector-Jacobian product of one molecule step (exact two-level, and RK4 GKSL
  with ladder decay, dephasing and several substeps for 3 and 5 levels) against
  central differences of the forward molecule step (which the molecule tests pin to
  closed forms);
* the full gradient against central differences of the forward flux
  (Sec. IV spectra) for a coupled problem with CPML, a design box, a source and
  molecules (two-level and multilevel), with Drude, Lorentz and three-pole media.
"""
import numpy as np
import pytest

from paper_2512_06173_gb300 import workloads as W


def _dot_case(oracle_mod, prob, seed):
    rng = np.random.default_rng(seed)
    o = oracle_mod.OracleSim(prob)
    sh = o.shape
    npl = o.npole
    x = [rng.standard_normal(sh) for _ in range(6)]
    psi = [rng.standard_normal(sh) for _ in range(12)]
    pol = [rng.standard_normal(sh) for _ in range(6 * npl)]
    o.set_fields(x)
    o.set_psi(psi)
    o.set_poles(pol)
    o.step(1)
    Lx = np.concatenate([np.ravel(f) for f in o.fields() + o.psi() + o.poles()])
    y = rng.standard_normal((18 + 6 * npl,) + sh)
    o.adj_reset()
    o.set_adj_state(y)
    o.adj_field_step()
    LTy = o.adj_state().ravel()
    xv = np.concatenate([np.ravel(f) for f in x + psi + pol])
    a, b = Lx @ y.ravel(), xv @ LTy
    return abs(a - b) / abs(a)


def test_field_step_dot_product_cpml_periodic(oracle_mod):
    prob = W.Problem(13, 11, 12, 0.5, periodic=(False, True, False), pml=(3, 4, 0, 0, 2, 3))
    assert _dot_case(oracle_mod, prob, 0) < 1e-12


def test_field_step_dot_product_materials_drude_walls(oracle_mod):
    mat = np.zeros((12, 11, 13), np.uint8)
    mat[4:8, 3:7, 5:9] = 1
    mat[0:3, :, :] = 2
    prob = W.Problem(13, 11, 12, 0.5, periodic=(False, False, True), pml=(3, 2, 2, 3, 0, 0), mat=mat,
                     materials=[W.Material(), W.Material(eps_inf=1.5, wp=0.8, gamma=0.1),
                                W.Material(eps_inf=2.25)])
    assert _dot_case(oracle_mod, prob, 1) < 1e-12


def test_field_step_dot_product_lorentz_and_multipole(oracle_mod):
    """Lorentz poles (the restoring term and the polarisation update) and materials with
    three poles, next to a Drude material and CPML."""
    mat = np.zeros((12, 11, 13), np.uint8)
    mat[4:8, 3:7, 5:9] = 1
    mat[0:3, :, :] = 2
    mat[9:11, 2:9, 1:12] = 3
    prob = W.Problem(13, 11, 12, 0.5, periodic=(False, True, False), pml=(3, 2, 0, 0, 2, 2), mat=mat,
                     materials=[W.Material(), W.Material(eps_inf=1.5, wp=0.8, gamma=0.1),
                                W.Material(eps_inf=2.0, wp=0.5, gamma=0.05, omega0=0.4),
                                W.Material(eps_inf=1.2, wp=0.6, gamma=0.02, omega0=0.3,
                                           extra=((0.4, 0.05, 0.55), (0.3, 0.1, 0.0)))])
    assert _dot_case(oracle_mod, prob, 2) < 1e-12


def test_molecule_vjp_matches_central_differences(oracle_mod):
    rng = np.random.default_rng(3)
    mu = np.array([[[0, .3], [.3, 0]], [[0, -.2j], [.2j, 0]], [[0.1, 0.5], [0.5, -0.1]]])
    rho = np.array([[0.6, 0.3 + 0.1j], [0.3 - 0.1j, 0.4]])
    mol = W.pack_molecules([dict(n=2, pos=[6.3, 5.1, 6.7], sigma=1.0, gamma=0.7, H0=np.diag([0.0, 0.25]),
                                 mu=mu, rho=rho)])
    o = oracle_mod.OracleSim(W.Problem(13, 11, 12, 0.5, molecules=mol))
    Et = rng.standard_normal(3)
    X = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    X = X + X.conj().T
    mdb = rng.standard_normal(3)
    rb, Etb = o.mol_vjp(0, Et, rho, X, mdb)

    def F(E, r):
        o.set_rho(0, r)
        md = o.molecule_step(0, E)
        return np.sum((X.conj() * o.rho(0)).real) + md @ mdb

    h = 1e-6
    fd = np.array([(F(Et + h * e, rho) - F(Et - h * e, rho)) / (2 * h) for e in np.eye(3)])
    np.testing.assert_allclose(Etb, fd, rtol=0, atol=1e-8)
    for d in [np.array([[1, 0], [0, 0]]), np.array([[0, 1], [1, 0]]), np.array([[0, 1j], [-1j, 0]])]:
        fdr = (F(Et, rho + h * d) - F(Et, rho - h * d)) / (2 * h)
        assert abs(fdr - np.sum((rb.conj() * d).real)) < 1e-8


@pytest.mark.parametrize("n,nsub", [(3, 1), (5, 2), (2, 3)])
def test_rk4_molecule_vjp_matches_central_differences(oracle_mod, n, nsub):
    rng = np.random.default_rng(10 + n)
    mu = np.stack([W.random_hermitian(rng, n, 0.3) for _ in range(3)])
    c = rng.normal(size=n) + 1j * rng.normal(size=n)
    c /= np.linalg.norm(c)
    rho = 0.7 * np.outer(c, c.conj()) + 0.3 * np.eye(n) / n
    E = np.concatenate([[0.0], np.cumsum(0.2 + 0.05 * rng.uniform(size=n - 1))])
    mol = W.pack_molecules([dict(n=n, pos=[6.3, 5.1, 6.7], sigma=1.0, gamma=0.7, H0=np.diag(E).astype(complex),
                                 mu=mu, rho=rho, decay=0.05, dephase=0.03, kind=W.KIND_RK4, nsub=nsub)])
    o = oracle_mod.OracleSim(W.Problem(13, 11, 12, 0.5, molecules=mol))
    Et = rng.standard_normal(3)
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    X = X + X.conj().T
    mdb = rng.standard_normal(3)
    rb, Etb = o.mol_vjp(0, Et, rho, X, mdb)

    def F(Ev, r):
        o.set_rho(0, r)
        md = o.molecule_step(0, Ev)
        return np.sum((X.conj() * o.rho(0)).real) + md @ mdb

    h = 1e-6
    fd = np.array([(F(Et + h * e, rho) - F(Et - h * e, rho)) / (2 * h) for e in np.eye(3)])
    np.testing.assert_allclose(Etb, fd, rtol=0, atol=1e-7)
    for _ in range(4):  # random Hermitian directions in rho
        d = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        d = d + d.conj().T
        fdr = (F(Et, rho + h * d) - F(Et, rho - h * d)) / (2 * h)
        assert abs(fdr - np.sum((rb.conj() * d).real)) < 1e-7


def _coupled(seed, drude=False, multilevel=False, lorentz=False):
    rng = np.random.default_rng(seed)
    nx, ny, nz = 14, 12, 20
    mats = [W.tls([rng.uniform(5, 9), rng.uniform(5, 7), rng.uniform(11, 13)], 0.3, 0.8, axis=q % 3,
                  sigma=0.8, gamma=rng.uniform(0.5, 1.5), cg=np.sqrt(0.7), ce=np.sqrt(0.3)) for q in range(3)]
    if multilevel:
        # RK4 GKSL systems of 3 and 4 levels with decay and dephasing, one with two substeps
        for q, n in enumerate((3, 4)):
            mu = np.stack([W.random_hermitian(rng, n, 0.4) for _ in range(3)])
            c = rng.normal(size=n) + 1j * rng.normal(size=n)
            c /= np.linalg.norm(c)
            E = np.concatenate([[0.0], np.cumsum(0.3 * (1 + 0.05 * rng.uniform(-1, 1, n - 1)))])
            mats.append(dict(n=n, pos=[rng.uniform(5, 9), rng.uniform(5, 7), rng.uniform(11, 13)], sigma=0.8,
                             gamma=rng.uniform(0.5, 1.5), H0=np.diag(E).astype(complex), mu=mu,
                             rho=np.outer(c, c.conj()), decay=0.02, dephase=0.01, kind=W.KIND_RK4, nsub=1 + q))
    mol = W.pack_molecules(mats)
    deps = 1.0 + rng.uniform(0, 1.5, (4, 5, 6))
    kw = {}
    if drude:
        m = np.zeros((nz, ny, nx), np.uint8)
        m[14:17, 2:6, 8:12] = 1
        mats = [W.Material(), W.Material(eps_inf=1.2, wp=0.9, gamma=0.05)]
        if lorentz:
            # a Lorentz oscillator and a three-pole material next to the Drude block
            m[14:17, 6:10, 8:12] = 2
            m[3:5, 2:10, 2:12] = 3
            mats += [W.Material(eps_inf=1.5, wp=0.5, gamma=0.02, omega0=0.3),
                     W.Material(eps_inf=1.1, wp=0.4, gamma=0.03, omega0=0.35,
                                extra=((0.3, 0.05, 0.5), (0.5, 0.08, 0.0)))]
        kw = dict(mat=m, materials=mats)
    return W.Problem(nx, ny, nz, 0.5, periodic=(False, True, False), pml=(3, 3, 0, 0, 3, 3),
                     design_box=(0 if drude else 4, 3, 6, 6, 5, 4), design_eps=deps,
                     sources=[W.Source(2, 4, 0, 1.0, 0.3, 6.0, 18.0)],
                     planes=[W.FluxPlane(2, 15, np.array([0.25, 0.3]))], molecules=mol, **kw)


@pytest.mark.parametrize("drude,multilevel,lorentz", [(False, False, False), (True, False, False),
                                                      (False, True, False), (True, False, True)])
def test_gradient_matches_central_differences(oracle_mod, drude, multilevel, lorentz):
    prob = _coupled(5, drude, multilevel, lorentz)
    NS = 80

    def J(p):
        o = oracle_mod.OracleSim(p)
        o.step(NS)
        return o.flux(0)[1]

    o = oracle_mod.OracleSim(prob)
    obj, ge, gg = o.adjoint_run(NS, 0, 1)
    assert obj == J(prob)
    x0, y0, z0 = prob.design_box[:3]
    h = 1e-4
    for (k, j, i) in [(6, 3, x0), (8, 5, x0 + 3), (9, 7, x0 + 5), (7, 4, x0 + 1)]:
        d2 = prob.design_eps.copy()
        d2[k - z0, j - y0, i - x0] += h
        d1 = prob.design_eps.copy()
        d1[k - z0, j - y0, i - x0] -= h
        fd = (J(prob.replace(design_eps=d2)) - J(prob.replace(design_eps=d1))) / (2 * h)
        assert abs(ge[k, j, i] - fd) <= 1e-6 * abs(fd)
    mol = prob.molecules
    for m in range(mol.count):
        g2, g1 = mol.gamma.copy(), mol.gamma.copy()
        g2[m] += h
        g1[m] -= h
        fd = (J(prob.replace(molecules=W.Molecules(mol.nlev, mol.off, mol.pos, mol.sigma, g2, mol.decay,
                                                    mol.dephase, mol.kind, mol.nsub, mol.H0, mol.mu, mol.rho0)))
              - J(prob.replace(molecules=W.Molecules(mol.nlev, mol.off, mol.pos, mol.sigma, g1, mol.decay,
                                                      mol.dephase, mol.kind, mol.nsub, mol.H0, mol.mu,
                                                      mol.rho0)))) / (2 * h)
        assert abs(gg[m] - fd) <= 1e-6 * abs(fd)
