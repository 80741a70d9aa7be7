"""FP64 oracle of laser-driven molecules in the classical-path approximation (test
infrastructure).

Only `tests/`, `__graft_entry__.smoke()` and the CPU legs of `bench.py` may import
this module.  Sec. II ("Using analytical solutions of Maxwell's equations") drives
molecules by a prescribed field with no back-action; in 1D vacuum a wave travelling
along z is a function of z - c t (Eq. E_analytical).  The waveform (a reading; the
paper leaves it open) is a carrier under an envelope of compact support:

    E~_m(t) = gamma_m E0 e_pol env(u) cos(k u + phase),  u = z_m - xi0 - c t,
    env(u) = cos^2(pi u / (2 W)) for |u| < W, else 0,   c = 1, k = omega,

held over each molecule step from t = n dt (the grid coupling's reading); molecules
advance by the oracle's own propagator.

Pinned by `tests/test_oracle_laser.py`: a molecule placed k dt further along z sees
the same field k steps later, so from the ground state its populations repeat those
of the first molecule shifted by k steps, exactly; a weak resonant pulse leaves the
first-order, rotating-wave excitation (mu E0 W / 2)^2 (the envelope integrates to W).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

from . import OracleSim


class OracleLaser:
    def __init__(self, molecules, amplitude: float, omega: float, phase: float, center: float,
                 half_width: float, polarization: Sequence[float], dt: float):
        from paper_2512_06173_gb300.workloads import Problem  # problem description only
        self.mol = molecules
        M = molecules.count
        self.z = np.array(molecules.pos[:, 2], np.float64)
        host = dataclasses.replace(molecules, pos=np.full((M, 3), 4.0), sigma=np.full(M, 0.5))
        self.sim = OracleSim(Problem(8, 8, 8, 0.5, periodic=(True, True, True), molecules=host))
        self.E0, self.k, self.phase = float(amplitude), float(omega), float(phase)
        self.xi0, self.W, self.dt = float(center), float(half_width), float(dt)
        self.pol = np.array(polarization, np.float64)
        self.nstep = 0

    def field(self, m: int, n: int) -> np.ndarray:
        """Eq. E_analytical at molecule m for the step that starts at t = n dt, before gamma_m."""
        u = (self.z[m] - self.xi0) - n * self.dt
        if abs(u) >= self.W:
            return np.zeros(3)
        env = math.cos(math.pi * u / (2.0 * self.W)) ** 2
        return self.E0 * env * math.cos(self.k * u + self.phase) * self.pol

    def rho(self, m: int) -> np.ndarray:
        return self.sim.rho(m)

    def populations(self) -> np.ndarray:
        return np.array([np.real(np.diag(self.rho(m)))[:2] for m in range(self.mol.count)])

    def step(self, n: int = 1):
        for _ in range(n):
            for m in range(self.mol.count):
                self.sim.molecule_step(m, float(self.mol.gamma[m]) * self.field(m, self.nstep), self.dt)
            self.nstep += 1
