"""FP64 oracle of the single-mode cavity solver (test infrastructure).

Only `tests/`, `__graft_entry__.smoke()` and the CPU legs of `bench.py` may import
this module.  It restates, step by step, the classical normal-mode field of Sec. II
("Classical photonic dynamics in normal modes") in the single-mode limit the paper
implements:

- field Hamiltonian Eq. H_F_normalmode with one mode of frequency w_c per polarisation
  lambda = x, y and mode function f = e_lambda / sqrt(V), so sqrt(V) f = e_lambda;
- equation of motion Eq. eom_cavmd_a, q'' = -w_c^2 q - eps d, with the coupling
  eps = w_c / sqrt(V eps0) of Eq. varepsilon_cavmd (eps0 = 1) given directly;
- total dipole Eq. dklambda_def, d_lambda = sum_m gamma_m <mu_lambda^(m)>, with the
  same per-molecule coupling rescale gamma_m as the grid coupling (gamma_m = 1 is the
  paper's);
- field at molecule m, Eq. E_normalmode:
      E~_m = -gamma_m sum_lambda [eps q_lambda + (eps^2 / w_c^2) d_lambda] e_lambda.

One step n -> n+1 of length dt (the reading, as for the grid coupling): the molecules
advance over the step with E~^n held (built from q^n and d^n), by the oracle's own
molecule propagator; d^{n+1} follows from rho^{n+1}; q, p advance by velocity Verlet,
the first half kick with d^n and the second with d^{n+1}.

Pinned by `tests/test_oracle_cavity.py`: the empty cavity against the closed-form
solution of the Verlet recursion; N identical co-located molecules against one with
gamma = sqrt(N); the two polariton frequencies of a weakly excited emitter against the
roots of the linear-response dispersion relation; energy conservation, with a
sign-flipped coupling as the control.
"""
from __future__ import annotations

import dataclasses
from typing import Sequence

import numpy as np

from . import OracleSim


class OracleCavity:
    """Single-mode cavity (polarisations x and y) coupled to `molecules`."""

    def __init__(self, molecules, omega_c: float, coupling: float, dt: float,
                 q0: Sequence[float] = (0.0, 0.0), p0: Sequence[float] = (0.0, 0.0)):
        from paper_2512_06173_gb300.workloads import Problem  # problem description only
        self.mol = molecules
        M = molecules.count
        # A small periodic grid only hosts the molecules for the oracle's propagator;
        # the cavity never reads its field.
        host = dataclasses.replace(molecules, pos=np.full((M, 3), 4.0), sigma=np.full(M, 0.5))
        self.sim = OracleSim(Problem(8, 8, 8, 0.5, periodic=(True, True, True), molecules=host))
        self.wc = float(omega_c)
        self.eps = float(coupling)
        self.dt = float(dt)
        self.q = np.array(q0, np.float64)
        self.p = np.array(p0, np.float64)
        self.mu = [np.stack([molecules.matrix(molecules.mu[a], m) for a in range(3)]) for m in range(M)]
        self.H0 = [molecules.matrix(molecules.H0, m) for m in range(M)]
        self.d = self.dipole()
        self.nstep = 0

    # ---- state
    def rho(self, m: int) -> np.ndarray:
        return self.sim.rho(m)

    def mu_expect(self, m: int) -> np.ndarray:
        """<mu> = Re Tr(rho mu) for each Cartesian component."""
        r = self.rho(m)
        return np.array([np.real(np.trace(r @ self.mu[m][a])) for a in range(3)])

    def dipole(self) -> np.ndarray:
        """d_lambda = sum_m gamma_m <mu_lambda>, lambda = x, y (Eq. dklambda_def)."""
        d = np.zeros(2)
        for m in range(self.mol.count):
            d += float(self.mol.gamma[m]) * self.mu_expect(m)[:2]
        return d

    def field(self) -> np.ndarray:
        """Field of Eq. E_normalmode before the per-molecule gamma_m (z component 0)."""
        e = -(self.eps * self.q + self.eps ** 2 / self.wc ** 2 * self.d)
        return np.array([e[0], e[1], 0.0])

    def energy(self) -> float:
        """Mode energy of Eq. H_F_normalmode with the molecules' mean dipoles,
        1/2 p^2 + 1/2 w_c^2 (q + eps d / w_c^2)^2 per polarisation, plus sum_m Tr(rho H0)."""
        e = 0.5 * np.sum(self.p ** 2) + 0.5 * self.wc ** 2 * np.sum((self.q + self.eps * self.d / self.wc ** 2) ** 2)
        for m in range(self.mol.count):
            e += float(np.real(np.trace(self.rho(m) @ self.H0[m])))
        return float(e)

    def mode(self) -> np.ndarray:
        """(q_x, q_y, p_x, p_y, d_x, d_y)."""
        return np.concatenate([self.q, self.p, self.d])

    # ---- dynamics
    def force(self, q: np.ndarray, d: np.ndarray) -> np.ndarray:
        """Eq. eom_cavmd_a: -w_c^2 q - eps d."""
        return -self.wc ** 2 * q - self.eps * d

    def step(self, n: int = 1):
        for _ in range(n):
            E = self.field()
            for m in range(self.mol.count):
                self.sim.molecule_step(m, float(self.mol.gamma[m]) * E, self.dt)
            d_new = self.dipole()
            p_half = self.p + 0.5 * self.dt * self.force(self.q, self.d)
            q_new = self.q + self.dt * p_half
            self.p = p_half + 0.5 * self.dt * self.force(q_new, d_new)
            self.q = q_new
            self.d = d_new
            self.nstep += 1
