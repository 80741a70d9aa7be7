"""Pins of the classical-path (laser-driven) oracle, oracle/laser.py:

- translation: the field depends on z - c t only (Eq. E_analytical), so a molecule
  placed k dt further along z repeats, k steps later, the populations of one at z
  (both from the ground state, which the field-free steps before the pulse leave
  unchanged up to round-off);
- first-order, rotating-wave excitation by a weak resonant pulse: with
  H = H0 - E mu sigma_x, c_e = i mu integral E(t) e^{i w0 t} dt, and for the carrier
  cos(w0 t + ...) under an envelope that integrates to W, P_e = (mu E0 W / 2)^2; the
  scheme converges to it as dt shrinks;
- polarisation: a field perpendicular to the dipole excites nothing.
"""
import numpy as np
import pytest

from paper_2512_06173_gb300 import workloads as W


@pytest.fixture(scope="module")
def las():
    from oracle import laser
    return laser


def test_translation_in_z_is_a_delay(las):
    dt, k, Wp = 0.5, 37, 50.0
    mols = W.pack_molecules([W.tls((0.0, 0.0, z), 0.25, 0.8, axis=0, gamma=1.3) for z in (10.0, 10.0 + k * dt)])
    o = las.OracleLaser(mols, 0.02, 0.25, 0.4, -Wp, Wp, (1.0, 0.0, 0.0), dt)
    hist = []
    for _ in range(400):
        o.step()
        hist.append(o.populations())
    moved = max(abs(h[0, 1]) for h in hist)
    assert moved > 1e-3
    for n in range(400 - k):
        assert np.abs(hist[n + k][1] - hist[n][0]).max() < 1e-13


@pytest.mark.parametrize("dt,tol", [(0.5, 5e-3), (0.1, 5e-4)])
def test_weak_resonant_pulse_first_order(las, dt, tol):
    E0, Wp, mu = 1e-4, 200.0, 1.0
    mols = W.pack_molecules([W.tls((0.0, 0.0, 10.0), 0.25, mu, axis=0)])
    o = las.OracleLaser(mols, E0, 0.25, 0.0, -Wp, Wp, (1.0, 0.0, 0.0), dt)
    o.step(int((10.0 + 2 * Wp + 20.0) / dt))
    pe = o.populations()[0, 1]
    assert abs(pe / (mu * E0 * Wp / 2) ** 2 - 1.0) < tol


def test_perpendicular_polarisation_excites_nothing(las):
    mols = W.pack_molecules([W.tls((0.0, 0.0, 10.0), 0.25, 1.0, axis=0)])
    o = las.OracleLaser(mols, 0.05, 0.25, 0.0, -40.0, 40.0, (0.0, 1.0, 0.0), 0.5)
    o.step(200)
    assert o.populations()[0, 1] < 1e-30
