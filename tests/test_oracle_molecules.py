"""Pins of the oracle's molecular propagation (Eq. von-Neumann-tls, Eq. dipole_derivative).

Checked against: closed-form free precession; the Taylor-polynomial form that one
RK4 step of a linear ODE must equal; a Kronecker-product (superoperator) form of
the GKSL equation built independently with numpy; scipy's matrix exponential;
brute-force small-step integration of the same ODE; the RWA Rabi law; closed forms
of amplitude damping and pure dephasing.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from paper_2512_06173_gb300.workloads import (KIND_EXACT2, KIND_RK4, Problem, pack_molecules,
                                              random_hermitian, tls)


def molsim(oracle_mod, mols, n=12):
    prob = Problem(n, n, n, 0.5, periodic=(True, True, True), molecules=pack_molecules(mols))
    return oracle_mod.OracleSim(prob)


def T4(z):
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


def test_free_precession_exact(oracle_mod):
    cg, ce = np.sqrt(0.9), np.sqrt(0.1) * np.exp(0.3j)
    s = molsim(oracle_mod, [tls((6, 6, 6), 0.25, 0.1, cg=cg, ce=ce)])
    r0 = s.rho(0)
    for n in range(1, 1001):
        s.molecule_step(0, [0, 0, 0])
    r = s.rho(0)
    t = 1000 * 0.5
    assert abs(r[0, 1] - r0[0, 1] * np.exp(1j * 0.25 * t)) < 1e-12
    assert abs(r[1, 1] - r0[1, 1]) < 1e-12 and abs(r[0, 0] - r0[0, 0]) < 1e-12


@pytest.mark.parametrize("nsub", [1, 3])
def test_rk4_free_precession_closed_form(oracle_mod, nsub):
    s = molsim(oracle_mod, [tls((6, 6, 6), 0.25, 0.1, cg=np.sqrt(0.7), ce=np.sqrt(0.3),
                                kind=KIND_RK4, nsub=nsub)])
    r0 = s.rho(0)
    steps = 400
    for _ in range(steps):
        s.molecule_step(0, [0, 0, 0])
    h = 0.5 / nsub
    want = r0[0, 1] * T4(1j * 0.25 * h) ** (steps * nsub)
    assert abs(s.rho(0)[0, 1] - want) < 1e-13


def superop(H, Ls):
    """Column-stacking vec: vec(A X B) = (B^T kron A) vec(X)."""
    n = H.shape[0]
    I = np.eye(n)
    L = -1j * (np.kron(I, H) - np.kron(H.T, I))
    for Lk in Ls:
        LdL = Lk.conj().T @ Lk
        L += np.kron(Lk.conj(), Lk) - 0.5 * np.kron(I, LdL) - 0.5 * np.kron(LdL.T, I)
    return L


def jump_ops(n, decay, deph):
    Ls = []
    for k in range(1, n):
        L = np.zeros((n, n), complex)
        L[k - 1, k] = np.sqrt(decay)
        Ls.append(L)
    for k in range(n):
        L = np.zeros((n, n), complex)
        L[k, k] = np.sqrt(deph)
        Ls.append(L)
    return Ls


def random_mol(rng, n):
    E = np.sort(rng.uniform(0, 1.5, n))
    mu = np.stack([random_hermitian(rng, n, 0.5) for _ in range(3)])
    c = rng.normal(size=n) + 1j * rng.normal(size=n)
    c /= np.linalg.norm(c)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    rho = A @ A.conj().T
    rho /= np.trace(rho)
    return dict(n=n, pos=(6, 6, 6), sigma=1.0, gamma=1.0, H0=np.diag(E) + random_hermitian(rng, n, 0.05),
                mu=mu, rho=rho, decay=float(rng.uniform(0, 0.1)), dephase=float(rng.uniform(0, 0.1)),
                kind=KIND_RK4, nsub=int(rng.integers(1, 4)))


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_lindblad_rhs_matches_superoperator(oracle_mod, n):
    rng = np.random.Generator(np.random.PCG64(n))
    d = random_mol(rng, n)
    s = molsim(oracle_mod, [d])
    Et = rng.normal(size=3)
    H = d["H0"] - sum(Et[a] * d["mu"][a] for a in range(3))
    L = superop(H, jump_ops(n, d["decay"], d["dephase"]))
    rho = d["rho"]
    want = (L @ rho.reshape(-1, order="F")).reshape(n, n, order="F")
    got = s.lindblad_rhs(0, Et, rho)
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("n", [2, 4, 8])
def test_rk4_step_equals_taylor_polynomial(oracle_mod, n):
    rng = np.random.Generator(np.random.PCG64(10 + n))
    d = random_mol(rng, n)
    s = molsim(oracle_mod, [d])
    Et = rng.normal(size=3) * 0.3
    H = d["H0"] - sum(Et[a] * d["mu"][a] for a in range(3))
    L = superop(H, jump_ops(n, d["decay"], d["dephase"]))
    h = 0.5 / d["nsub"]
    P = sum(np.linalg.matrix_power(h * L, j) / math.factorial(j) for j in range(5))
    v = d["rho"].reshape(-1, order="F")
    for _ in range(d["nsub"]):
        v = P @ v
    s.molecule_step(0, Et)
    assert np.abs(s.rho(0) - v.reshape(n, n, order="F")).max() < 1e-13


def test_exact2_matches_expm(oracle_mod):
    rng = np.random.Generator(np.random.PCG64(5))
    d = tls((6, 6, 6), 0.37, 0.8, axis=1, cg=0.6, ce=0.8j)
    d["H0"] = np.array([[0.1, 0.05 - 0.02j], [0.05 + 0.02j, 0.45]])
    d["mu"][0] = random_hermitian(rng, 2, 0.3)
    d["kind"] = KIND_EXACT2
    s = molsim(oracle_mod, [d])
    rho = s.rho(0)
    for _ in range(25):
        Et = rng.normal(size=3)
        H = d["H0"] - sum(Et[a] * d["mu"][a] for a in range(3))
        U = sla.expm(-1j * H * 0.5)
        rho = U @ rho @ U.conj().T
        s.molecule_step(0, Et)
    assert np.abs(s.rho(0) - rho).max() < 1e-13


def brute_force(H0, mu, rho, fields, dt, sub=400):
    """Fine-step RK4 of drho/dt = -i[H0 - E mu, rho] with the field held per step."""
    h = dt / sub
    for E in fields:
        H = H0 - E * mu

        def f(r):
            return -1j * (H @ r - r @ H)

        for _ in range(sub):
            k1 = f(rho); k2 = f(rho + h / 2 * k1); k3 = f(rho + h / 2 * k2); k4 = f(rho + h * k3)
            rho = rho + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return rho


def test_rabi_against_brute_force_and_rwa(oracle_mod):
    w0, mu12, E0, dt = 0.25, 0.1, 0.05, 0.5
    s = molsim(oracle_mod, [tls((6, 6, 6), w0, mu12, axis=2, cg=1.0, ce=0.0)])
    steps = 2513  # about one Rabi period 2 pi / (mu12 E0) at dt = 0.5
    fields = [E0 * np.cos(w0 * n * dt) for n in range(steps)]
    pe = []
    for E in fields:
        s.molecule_step(0, [0, 0, E])
        pe.append(s.rho(0)[1, 1].real)
    # the exact propagator against brute force on the first 300 steps
    H0 = np.diag([0, w0]).astype(complex)
    mu = mu12 * np.array([[0, 1], [1, 0]], complex)
    r_bf = brute_force(H0, mu, np.diag([1, 0]).astype(complex), fields[:300], dt)
    s2 = molsim(oracle_mod, [tls((6, 6, 6), w0, mu12, axis=2, cg=1.0, ce=0.0)])
    for E in fields[:300]:
        s2.molecule_step(0, [0, 0, E])
    assert np.abs(s2.rho(0) - r_bf).max() < 1e-10
    # rotating-wave law P_e = sin^2(mu E0 t / 2), error O(mu E0 / w0)
    t = (np.arange(steps) + 1) * dt
    rwa = np.sin(mu12 * E0 * t / 2) ** 2
    assert np.abs(np.array(pe) - rwa).max() < 0.03
    assert max(pe) > 0.97


def test_amplitude_damping_cascade(oracle_mod):
    G, dt = 0.01, 0.5
    rho = np.zeros((3, 3), complex)
    rho[2, 2] = 1
    d = dict(n=3, pos=(6, 6, 6), sigma=1.0, gamma=1.0, H0=np.diag([0, 0.2, 0.41]).astype(complex),
             mu=np.zeros((3, 3, 3)), rho=rho, decay=G, dephase=0.0, kind=KIND_RK4, nsub=1)
    s = molsim(oracle_mod, [d])
    steps = 600
    for _ in range(steps):
        s.molecule_step(0, [0, 0, 0])
    t = steps * dt
    p = np.real(np.diag(s.rho(0)))
    want = [1 - np.exp(-G * t) - G * t * np.exp(-G * t), G * t * np.exp(-G * t), np.exp(-G * t)]
    assert np.abs(p - want).max() < 1e-9


def test_pure_dephasing_closed_form(oracle_mod):
    g, w0 = 0.02, 0.25
    s = molsim(oracle_mod, [tls((6, 6, 6), w0, 0.0, cg=np.sqrt(0.5), ce=np.sqrt(0.5),
                                dephase=g, kind=KIND_RK4, nsub=2)])
    r0 = s.rho(0)
    steps = 300
    for _ in range(steps):
        s.molecule_step(0, [0, 0, 0])
    r = s.rho(0)
    h = 0.25
    assert abs(r[0, 1] - r0[0, 1] * T4((1j * w0 - g) * h) ** (2 * steps)) < 1e-13
    assert abs(abs(r[0, 1]) - 0.5 * np.exp(-g * steps * 0.5)) < 1e-6  # RK4 truncation
    assert abs(r[1, 1] - 0.5) < 1e-14


def test_trace_and_hermiticity(oracle_mod):
    rng = np.random.Generator(np.random.PCG64(99))
    ds = [random_mol(rng, n) for n in (2, 5, 8)]
    s = molsim(oracle_mod, ds)
    for _ in range(200):
        for m in range(3):
            s.molecule_step(m, rng.normal(size=3) * 0.2)
    for m in range(3):
        r = s.rho(m)
        assert abs(np.trace(r) - 1) < 1e-12
        assert np.abs(r - r.conj().T).max() < 1e-14
        assert np.linalg.eigvalsh(r).min() > -1e-10


def test_dipole_derivative_identity(oracle_mod):
    """Tr(drho/dt mu) = -2 w0 mu01 Im(rho01) e_i for the dissipation-free two-level
    system (the analytic form given after Eq. dipole_derivative), and the finite
    difference used by the step converges to it at second order."""
    w0, mu12 = 0.25, 0.3
    s = molsim(oracle_mod, [tls((6, 6, 6), w0, mu12, axis=0, cg=0.8, ce=0.6 * np.exp(0.7j),
                                kind=KIND_RK4)])
    rho = s.rho(0)
    Et = np.array([0.04, 0.0, 0.0])
    rd = s.lindblad_rhs(0, Et, rho)
    mu = mu12 * np.array([[0, 1], [1, 0]])
    assert abs(np.trace(rd @ mu).real - (-2 * w0 * mu12 * rho[0, 1].imag)) < 1e-15
    errs = []
    for dt in (0.2, 0.1):
        s2 = molsim(oracle_mod, [tls((6, 6, 6), w0, mu12, axis=0, cg=0.8, ce=0.6 * np.exp(0.7j),
                                     kind=KIND_EXACT2)])
        md = s2.molecule_step(0, Et, dt)[0]
        rm = s2.rho(0)
        # analytic rate at the midpoint of the step
        mid = (rho + rm) / 2
        errs.append(abs(md - (-2 * w0 * mu12 * mid[0, 1].imag)))
    assert errs[1] < errs[0] / 3.5


def test_energy_sum_free_precession(oracle_mod):
    """The per-molecule energy accumulator sums Tr(rho^{n+1} H0) over steps; for an
    uncoupled emitter Tr(rho H0) = w0 rho_11 stays constant, so after N steps the sum
    is N w0 rho_11 (and the multilevel ladder gives sum_k E_k rho_kk)."""
    w0 = 0.31
    d = tls((3.3, 3.7, 3.1), w0, 0.0, cg=np.sqrt(0.6), ce=np.sqrt(0.4) * np.exp(0.2j))
    rho = np.diag([0.5, 0.3, 0.2]).astype(complex)
    d3 = dict(n=3, pos=(4.2, 3.1, 2.9), sigma=1.0, gamma=1.0, H0=np.diag([0.0, 0.2, 0.45]).astype(complex),
              mu=np.zeros((3, 3, 3)), rho=rho, kind=KIND_RK4, nsub=1)
    prob = Problem(8, 8, 8, 0.5, periodic=(True, True, True), molecules=pack_molecules([d, d3]))
    s = oracle_mod.OracleSim(prob)
    s.step(37)
    assert abs(s.mol_state(0)[2] - 37 * w0 * 0.4) < 1e-12
    assert abs(s.mol_state(1)[2] - 37 * (0.2 * 0.3 + 0.45 * 0.2)) < 1e-12
