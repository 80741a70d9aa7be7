"""Pins of the single-mode cavity oracle (oracle/cavity.py) by facts it does not
compute itself:

- empty cavity: velocity Verlet on q'' = -w^2 q is the recursion
  q^{n+1} - 2 q^n + q^{n-1} = -w^2 dt^2 q^n, solved in closed form by
  q^n = q0 cos(W n dt) + (dt p0 / sin(W dt)) sin(W n dt), cos(W dt) = 1 - w^2 dt^2 / 2;
- N identical co-located molecules with gamma = 1 against one molecule with
  gamma = sqrt(N) from an empty mode: identical density matrices, q scaled by sqrt(N);
- polaritons: a weakly excited two-level emitter resonant with the mode; the spectrum
  of q(t) peaks at the roots of the linear-response dispersion relation
  (w_c^2 - w^2)(w0^2 - w^2) w_c^2 = 2 gamma^2 mu^2 w0 eps^2 w^2
  (two-level polarisability 2 mu^2 w0 / (w0^2 - w^2), with the dipole self-energy term);
- energy: 1/2 p^2 + 1/2 w_c^2 (q + eps d / w_c^2)^2 + sum Tr(rho H0), conserved by the
  exact dynamics without dissipation, drifts at first order in dt (the field is held
  over each molecule step); with the coupling's sign flipped in the field (a plausible
  mistake) the drift does not shrink with dt.
"""
import numpy as np
import pytest

from paper_2512_06173_gb300 import workloads as W


@pytest.fixture(scope="module")
def cav():
    from oracle import cavity
    return cavity


def tls(**kw):
    return W.tls((4.0, 4.0, 4.0), **kw)


def test_empty_cavity_is_the_verlet_oscillator(cav):
    wc, dt = 0.3, 0.5
    q0, p0 = np.array([0.7, -0.2]), np.array([0.1, 0.4])
    c = cav.OracleCavity(W.empty_molecules(), wc, 0.05, dt, q0=q0, p0=p0)
    Wd = np.arccos(1.0 - 0.5 * wc ** 2 * dt ** 2) / dt
    for n in range(1, 801):
        c.step()
        want = q0 * np.cos(Wd * n * dt) + dt * p0 / np.sin(Wd * dt) * np.sin(Wd * n * dt)
        assert np.abs(c.q - want).max() < 1e-11


@pytest.mark.parametrize("dephase", [0.0, 2e-3])
def test_copies_equal_one_molecule_with_sqrt_n_coupling(cav, dephase):
    N = 5
    kw = dict(omega0=0.25, mu12=0.8, axis=0, cg=np.sqrt(0.6), ce=np.sqrt(0.4) * np.exp(0.3j), dephase=dephase)
    many = cav.OracleCavity(W.pack_molecules([tls(**kw) for _ in range(N)]), 0.25, 0.02, 0.5)
    one = cav.OracleCavity(W.pack_molecules([tls(gamma=np.sqrt(N), **kw)]), 0.25, 0.02, 0.5)
    for _ in range(300):
        many.step()
        one.step()
    for m in range(N):
        assert np.abs(many.rho(m) - one.rho(0)).max() < 1e-12
    assert np.abs(many.q - np.sqrt(N) * one.q).max() < 1e-11 * max(1.0, np.abs(many.q).max())


def test_polariton_frequencies(cav):
    # The field is held over each molecule step, so the coupled linear system gains
    # energy at a rate of order g^2 dt (g the coupling frequency); dt = 0.1 keeps that
    # growth below a factor 2 over the run and the emitter in the linear regime.
    w0 = wc = 0.25
    mu, gam, eps, dt, steps = 1.0, 2.0, 0.004, 0.1, 100000
    c = cav.OracleCavity(W.pack_molecules([tls(omega0=w0, mu12=mu, axis=0, gamma=gam, cg=np.sqrt(1 - 1e-8),
                                               ce=1e-4)]), wc, eps, dt)
    qs = np.empty(steps)
    for n in range(steps):
        c.step()
        qs[n] = c.q[0]
    # closed form: roots in w^2 of (wc^2 - w^2)(w0^2 - w^2) wc^2 - 2 gam^2 mu^2 w0 eps^2 w^2 = 0
    k = 2 * gam ** 2 * mu ** 2 * w0 * eps ** 2 / wc ** 2
    roots = np.sort(np.sqrt(np.roots([1.0, -(wc ** 2 + w0 ** 2 + k), wc ** 2 * w0 ** 2]).real))
    # spectrum with a Hann window; peaks refined by a parabola through the log magnitude
    x = (qs - qs.mean()) * np.hanning(steps)
    nfft = 1 << 20
    S = np.abs(np.fft.rfft(x, nfft))
    w = 2 * np.pi * np.fft.rfftfreq(nfft, dt)
    band = (w > 0.15) & (w < 0.35)
    idx = np.where(band)[0]
    loc = [i for i in idx[1:-1] if S[i] > S[i - 1] and S[i] >= S[i + 1]]
    loc = sorted(sorted(loc, key=lambda i: -S[i])[:2])
    peaks = []
    for i in loc:
        a, b, cc = np.log(S[i - 1]), np.log(S[i]), np.log(S[i + 1])
        peaks.append(w[i] + 0.5 * (a - cc) / (a - 2 * b + cc) * (w[1] - w[0]))
    assert len(peaks) == 2
    split = roots[1] - roots[0]
    assert split > 0.05 * w0  # a resolved splitting, not a single peak
    assert np.abs(np.array(peaks) - roots).max() < 0.03 * split


def energy_drift(cav, dt, flip):
    mols = W.pack_molecules([tls(omega0=0.25, mu12=1.0, axis=a % 2, gamma=1.0 + 0.5 * a) for a in range(3)])
    c = cav.OracleCavity(mols, 0.25, 0.02, dt, q0=(2.0, -1.0), p0=(0.0, 0.5))
    if flip:  # the plausible sign mistake in Eq. E_normalmode
        base = c.field
        c.field = lambda: -base()
    e0 = c.energy()
    mol_e = lambda: sum(float(np.real(np.trace(c.rho(m) @ c.H0[m]))) for m in range(mols.count))
    m0 = mol_e()
    drift, moved = 0.0, 0.0
    for _ in range(int(round(200 / dt))):
        c.step()
        drift = max(drift, abs(c.energy() - e0))
        moved = max(moved, abs(mol_e() - m0))
    return drift, moved


def test_energy_conservation_to_first_order(cav):
    """With the field held over each molecule step the coupling is first order in dt:
    the energy error halves with dt; with the coupling's sign flipped it does not
    shrink at all."""
    d1, moved = energy_drift(cav, 0.1, False)
    d2, _ = energy_drift(cav, 0.05, False)
    assert moved > 0.1  # energy does flow between the mode and the emitters
    assert 1.7 < d1 / d2 < 2.5
    assert d2 < 0.05 * moved
    f1, _ = energy_drift(cav, 0.1, True)
    f2, _ = energy_drift(cav, 0.05, True)
    assert f2 > 0.9 * f1 and f2 > moved
