"""Pins of the oracle's DFT flux planes and Drude medium.

  * DFT accumulators of a travelling Yee eigenmode equal the closed-form sums of the
    analytic field (E sampled at t = (n+1) dt, H at (n+1/2) dt, weight dt), and the
    flux assembled from them equals the closed form and is positive along +k.
  * A current sheet in a box periodic in x, y: equal flux through two planes on the
    same side, equal and opposite flux on the two sides.
  * Drude ADE: a spatially uniform field in a Drude medium oscillates as the damped
    plasma oscillation E(t) = E0 e^{-g t/2}(cos w't + g/(2w') sin w't), w'^2 = wp^2/eps - g^2/4.
  * Lorentz pole: the same oscillation about the shifted equilibrium; several poles in
    one cell: the exact solution of the continuous uniform-field equations (matrix
    exponential), energy bookkeeping over all poles, and two half-strength poles equal
    to one full-strength pole.
  * Poynting closure: the energy a dispersive layer absorbs (time-domain work on its
    poles) equals the net DFT flux into it integrated over frequency (Parseval), to
    second order in dt.
"""
import numpy as np
import pytest

from paper_2512_06173_gb300.workloads import FluxPlane, Material, Problem, Source

from test_oracle_yee import eigenmode


def test_dft_accumulators_of_eigenmode(oracle_mod):
    shape = (16, 6, 5)  # nz, ny, nx
    dt = 0.5
    om = np.array([0.31, 0.5, 0.77])
    prob = Problem(5, 6, 16, dt, periodic=(True, True, True), planes=[FluxPlane(2, 7, om)])
    sim = oracle_mod.OracleSim(prob)
    e_dir = np.array([0.0, 1.0, 0.0])
    f0, w = eigenmode(shape, (0, 0, 1), dt, 0.0, e_dir)
    sim.set_fields(f0)
    N = 137
    sim.step(N)
    E1, E2, H1, H2 = sim.plane_data(0)
    wantE = [np.zeros((3, 6, 5), complex) for _ in range(2)]
    wantH = [np.zeros((3, 6, 5), complex) for _ in range(2)]
    for n in range(N):
        fe, _ = eigenmode(shape, (0, 0, 1), dt, (n + 1) * dt, e_dir)
        # fields at t_E=(n+1)dt; H returned at t_E - dt/2 = (n+1/2) dt
        for fi in range(3):
            pe = np.exp(1j * om[fi] * (n + 1) * dt) * dt
            ph = np.exp(1j * om[fi] * (n + 0.5) * dt) * dt
            wantE[0][fi] += pe * fe[0][7]
            wantE[1][fi] += pe * fe[1][7]
            wantH[0][fi] += ph * 0.5 * (fe[3][7] + fe[3][6])
            wantH[1][fi] += ph * 0.5 * (fe[4][7] + fe[4][6])
    for got, want in zip([E1, E2, H1, H2], wantE + wantH):
        assert np.abs(got - want).max() < 1e-11
    flux = sim.flux(0)
    want_flux = np.array([np.real(wantE[0][f] * np.conj(wantH[1][f]) - wantE[1][f] * np.conj(wantH[0][f])).sum()
                          for f in range(3)])
    assert np.allclose(flux, want_flux, rtol=1e-11, atol=1e-12)
    # a +z wave carries positive flux at its own frequency
    p2 = Problem(5, 6, 16, dt, periodic=(True, True, True), planes=[FluxPlane(2, 7, np.array([w]))])
    s2 = oracle_mod.OracleSim(p2)
    s2.set_fields(f0)
    s2.step(400)
    assert s2.flux(0)[0] > 0


def test_sheet_source_flux_balance(oracle_mod):
    om = np.array([0.2, 0.3, 0.4])
    nz = 96
    planes = [FluxPlane(2, 60, om), FluxPlane(2, 75, om), FluxPlane(2, 30, om)]
    prob = Problem(4, 4, nz, 0.5, periodic=(True, True, False), pml=(0, 0, 0, 0, 12, 12),
                   sources=[Source(2, 48, 0, 1.0, 0.3, 6.0, 30.0)], planes=planes)
    sim = oracle_mod.OracleSim(prob)
    sim.step(900)
    f1, f2, f3 = sim.flux(0), sim.flux(1), sim.flux(2)
    assert np.all(f1 > 0) and np.all(f3 < 0)
    assert np.allclose(f1, f2, rtol=2e-3)
    assert np.allclose(f1, -f3, rtol=2e-3)


def test_drude_plasma_oscillation(oracle_mod):
    wp, g, einf, dt = 1.0, 0.05, 1.0, 0.002
    prob = Problem(3, 3, 3, dt, periodic=(True, True, True), mat=np.zeros((3, 3, 3), np.uint8),
                   materials=[Material(einf, wp, g)])
    sim = oracle_mod.OracleSim(prob)
    E0 = 0.7
    sim.set_fields([np.full((3, 3, 3), E0), np.zeros((3, 3, 3)), np.zeros((3, 3, 3))] +
                   [np.zeros((3, 3, 3))] * 3)
    ws = np.sqrt(wp ** 2 / einf - g ** 2 / 4)
    maxerr = 0.0
    for n in range(1, 15001):
        sim.step(1)
        t = n * dt
        want = E0 * np.exp(-g * t / 2) * (np.cos(ws * t) + g / (2 * ws) * np.sin(ws * t))
        maxerr = max(maxerr, abs(sim.fields()[0][1, 1, 1] - want))
    # the half-step Drude current starts at 0 instead of J(-dt/2): O(wp dt / 2) amplitude
    # error; the frequency error is O((wp dt)^2)
    assert maxerr < 2e-3 * E0
    # energy bookkeeping: the accumulated work sum J_D . (E^n + E^{n+1})/2 dt on the
    # Drude current plus the field energy stays at the initial field energy
    Ef = sim.fields()[0]
    tot = 0.5 * einf * (Ef ** 2).sum() + sim.absorbed()
    assert abs(tot - 0.5 * einf * E0 ** 2 * 27) < 2e-3 * 0.5 * E0 ** 2 * 27


def test_lorentz_oscillation(oracle_mod):
    """A uniform field in a Lorentz medium (no curl): eps_inf E' = -J, J' = -g J - w0^2 P
    + wp^2 E, P' = J conserve eps_inf E + P, so E'' + g E' + W^2 E = w0^2 E0 with
    W^2 = w0^2 + wp^2 / eps_inf: a damped oscillation at sqrt(W^2 - g^2/4) about the
    shifted equilibrium w0^2 E0 / W^2 (0 for a Drude pole), and the field energy plus the
    work done on the medium stays at the initial field energy."""
    wp, g, einf, w0, dt = 0.8, 0.05, 2.0, 0.6, 0.002
    prob = Problem(3, 3, 3, dt, periodic=(True, True, True), mat=np.zeros((3, 3, 3), np.uint8),
                   materials=[Material(einf, wp, g, w0)])
    sim = oracle_mod.OracleSim(prob)
    E0 = 0.7
    sim.set_fields([np.full((3, 3, 3), E0), np.zeros((3, 3, 3)), np.zeros((3, 3, 3))] +
                   [np.zeros((3, 3, 3))] * 3)
    W2 = w0 ** 2 + wp ** 2 / einf
    ws = np.sqrt(W2 - g ** 2 / 4)
    Eeq = w0 ** 2 * E0 / W2
    maxerr = 0.0
    for n in range(1, 15001):
        sim.step(1)
        t = n * dt
        want = Eeq + (E0 - Eeq) * np.exp(-g * t / 2) * (np.cos(ws * t) + g / (2 * ws) * np.sin(ws * t))
        maxerr = max(maxerr, abs(sim.fields()[0][1, 1, 1] - want))
    assert maxerr < 2e-3 * E0
    Ef = sim.fields()[0]
    tot = 0.5 * einf * (Ef ** 2).sum() + sim.absorbed()
    assert abs(tot - 0.5 * einf * E0 ** 2 * 27) < 2e-3 * 0.5 * einf * E0 ** 2 * 27


def _two_pole_uniform(oracle_mod, dt, T=20.0):
    """Oracle E(t) in a uniform field against the exact solution of the continuous
    equations eps_inf E' = -(J1 + J2), J_p' = -g_p J_p - w0_p^2 P_p + wp_p^2 E, P_p' = J_p
    (x' = A x, solved by the matrix exponential), for a Drude pole plus a Lorentz pole."""
    from scipy.linalg import expm
    einf = 1.5
    poles = [(0.5, 0.03, 0.0), (0.7, 0.05, 0.9)]
    prob = Problem(3, 3, 3, dt, periodic=(True, True, True), mat=np.zeros((3, 3, 3), np.uint8),
                   materials=[Material(einf, *poles[0], extra=(poles[1],))])
    sim = oracle_mod.OracleSim(prob)
    E0 = 0.7
    sim.set_fields([np.full((3, 3, 3), E0)] + [np.zeros((3, 3, 3))] * 5)
    A = np.zeros((5, 5))  # state (E, J1, P1, J2, P2)
    for p, (wp, g, w0) in enumerate(poles):
        j, q = 1 + 2 * p, 2 + 2 * p
        A[0, j] = -1.0 / einf
        A[j, j], A[j, q], A[j, 0], A[q, j] = -g, -w0 ** 2, wp ** 2, 1.0
    x0 = np.array([E0, 0.0, 0.0, 0.0, 0.0])
    err = 0.0
    n = int(round(T / dt))
    for s in range(1, n + 1):
        sim.step(1)
        if s % 50 == 0:
            err = max(err, abs(sim.fields()[0][1, 1, 1] - (expm(A * s * dt) @ x0)[0]))
    Ef = sim.fields()[0]
    e_init = 0.5 * einf * E0 ** 2 * 27
    return err, abs(0.5 * einf * (Ef ** 2).sum() + sim.absorbed() - e_init) / e_init


def test_two_pole_medium_against_the_continuous_solution(oracle_mod):
    """Drude + Lorentz poles in one cell: the scheme converges (first order, from the
    staggered start J^{-1/2} = 0) to the exact uniform-field solution, and the field
    energy plus the work done on both poles stays at the initial field energy."""
    e1, b1 = _two_pole_uniform(oracle_mod, 0.004)
    e2, b2 = _two_pole_uniform(oracle_mod, 0.002)
    assert e1 < 1.5e-3 * 0.7
    assert 1.8 < e1 / e2 < 2.2
    assert max(b1, b2) < 1e-12


def test_split_pole_equals_one_pole(oracle_mod):
    """The pole ADE is linear in wp^2: two identical poles of strength wp / sqrt(2)
    carry together the current of one pole of strength wp, in a 3D run with CPML,
    a source and a Lorentz sphere."""
    def prob(mat):
        n = 14
        zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        m = (((xx - 6.5) ** 2 + (yy - 7) ** 2 + (zz - 7.5) ** 2) < 16).astype(np.uint8)
        return Problem(n, n, n, 0.5, pml=(3,) * 6, mat=m, materials=[Material(1.0), mat],
                       sources=[Source(axis=2, index=4, comp=0, amp=1.0, omega=0.6, width=3.0, t0=8.0)])
    wp, g, w0 = 0.9, 0.04, 0.6
    a = oracle_mod.OracleSim(prob(Material(1.3, wp, g, w0)))
    h = wp / np.sqrt(2.0)
    b = oracle_mod.OracleSim(prob(Material(1.3, h, g, w0, extra=((h, g, w0),))))
    a.step(80)
    b.step(80)
    fa, fb = a.fields(), b.fields()
    scale = max(np.abs(f).max() for f in fa)
    assert scale > 1e-3
    for x, y in zip(fa, fb):
        assert np.abs(x - y).max() < 1e-12 * scale
    assert abs(a.absorbed() - b.absorbed()) < 1e-12 * abs(a.absorbed())


def _closure(oracle_mod, dt, materials):
    """Energy absorbed by a dispersive layer, two ways: the oracle's time-domain work on
    the poles, and the net DFT flux into the layer integrated over frequency (Parseval:
    integral of E x H over time = (1/pi) integral over w > 0 of Re(E~ x H~*))."""
    nz = 200
    mat = np.zeros((nz, 1, 1), np.uint8)
    mat[90:96] = 1
    om = np.linspace(0.0, 0.7, 281)  # the pulse's spectrum is negligible above 0.7
    p = Problem(1, 1, nz, dt, periodic=(True, True, False), pml=(0, 0, 0, 0, 12, 12), mat=mat,
                materials=materials,
                sources=[Source(axis=2, index=16, comp=0, amp=1.0, omega=0.25, width=12.0, t0=72.0)],
                planes=[FluxPlane(2, 60, om), FluxPlane(2, 130, om)])
    sim = oracle_mod.OracleSim(p)
    sim.step(int(round(1500 / dt)))
    trap = getattr(np, "trapezoid", None) or getattr(np, "trapz")
    into = trap(sim.flux(0) - sim.flux(1), om) / np.pi
    return sim.absorbed(), into


def test_poynting_closure_of_an_absorbing_layer(oracle_mod):
    """A pulse through a 6-cell layer (1 x 1 periodic cross-section): the energy the
    poles absorbed equals the net flux into the layer, to second order in dt (E is
    sampled at whole steps, H at half steps), for a Drude layer and for a Drude + Lorentz
    layer (whose reversibly stored energy has rung down by the end of the run)."""
    drude = [Material(1.0), Material(1.0, 1.0, 0.05)]
    a1, f1 = _closure(oracle_mod, 0.5, drude)
    a2, f2 = _closure(oracle_mod, 0.25, drude)
    assert a1 > 0.1
    e1, e2 = abs(f1 / a1 - 1), abs(f2 / a2 - 1)
    assert e1 < 5e-3 and 3.0 < e1 / e2 < 5.0, (e1, e2)
    multi = [Material(1.0), Material(1.5, 0.6, 0.05, 0.3, extra=((0.5, 0.1, 0.0),))]
    a3, f3 = _closure(oracle_mod, 0.5, multi)
    assert a3 > 0.1 and abs(f3 / a3 - 1) < 5e-3
