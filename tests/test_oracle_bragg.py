"""Pin of the oracle's layered-dielectric transmission (the Bragg stack of the strong-
coupling example, Sec. IV.C) by a calculation that shares none of its code: the
normal-incidence transfer matrix of the discretised stack.

A 1 x 1 cross-section, periodic in x and y, reduces the 3D Yee grid exactly to the 1D
chain Ex(k), Hy(k+1/2). At frequency omega the leapfrog's time difference becomes
-i Omega with Omega = 2 sin(omega dt / 2) / dt, so a time-harmonic solution obeys

    H_k = H_{k-1} + i Omega eps_k E_k,    E_{k+1} = E_k + i Omega H_k,

whose vacuum solutions are exp(+-i kappa k) with 2 sin(kappa / 2) = Omega (the Yee
dispersion relation).  Imposing a purely outgoing wave behind the stack and propagating
back gives the incident amplitude A in front of it, and the power transmission is
1 / |A|^2 (vacuum on both sides).  The oracle's transmission is the far flux plane's
DFT flux with the stack over the same without it, for a Gaussian pulse from a current
sheet; CPML on the z faces.
"""
import numpy as np

from paper_2512_06173_gb300.workloads import FluxPlane, Material, Problem, Source

DT = 0.5
NZ = 260


def stack(eps_hi=2.25, periods=5, hi=4, lo=6, z0=80):
    """Quarter-wave stack at omega = 0.25 (n = 1.5: 4 cells; vacuum: 6 cells)."""
    eps = np.ones(NZ)
    z = z0
    for _ in range(periods):
        eps[z:z + hi] = eps_hi
        z += hi + lo
    return eps


def oracle_flux(oracle_mod, eps, om):
    levels = sorted(set(eps.tolist()))
    mat = np.array([levels.index(e) for e in eps], np.uint8).reshape(NZ, 1, 1)
    p = Problem(1, 1, NZ, DT, periodic=(True, True, False), pml=(0, 0, 0, 0, 12, 12), mat=mat,
                materials=[Material(e) for e in levels],
                sources=[Source(axis=2, index=16, comp=0, amp=1.0, omega=0.25, width=12.0, t0=72.0)],
                planes=[FluxPlane(2, NZ - 24, om)])
    o = oracle_mod.OracleSim(p)
    o.step(5000)
    return o.flux(0)


def transfer_matrix(eps, om):
    out = []
    for w in om:
        Om = 2.0 * np.sin(w * DT / 2.0) / DT
        kap = 2.0 * np.arcsin(Om / 2.0)
        # outgoing wave behind the stack: E_k = exp(i kap k), H_{k-1} = (E_k - E_{k-1}) / (i Om)
        k = len(eps)
        E = np.exp(1j * kap * k)
        Hm = (E - np.exp(1j * kap * (k - 1))) / (1j * Om)
        for kk in range(len(eps) - 1, -1, -1):  # (E_{kk+1}, H_kk) -> (E_kk, H_{kk-1})
            Hk = Hm
            E = E - 1j * Om * Hk
            Hm = Hk - 1j * Om * eps[kk] * E
        # in front: E_0 = A + B, H_{-1} = A (1 - e^{-i kap}) / (i Om) + B (1 - e^{i kap}) / (i Om)
        M = np.array([[1.0, 1.0], [(1 - np.exp(-1j * kap)) / (1j * Om), (1 - np.exp(1j * kap)) / (1j * Om)]])
        A, _ = np.linalg.solve(M, [E, Hm])
        out.append(1.0 / abs(A) ** 2)
    return np.array(out)


def test_bragg_stack_transmission_matches_the_transfer_matrix(oracle_mod):
    om = np.linspace(0.15, 0.35, 9)
    eps = stack()
    T = oracle_flux(oracle_mod, eps, om) / oracle_flux(oracle_mod, np.ones(NZ), om)
    want = transfer_matrix(eps, om)
    assert np.abs(transfer_matrix(np.ones(NZ), om) - 1.0).max() < 1e-12  # vacuum transmits all
    assert want.min() < 0.1  # the stop band is resolved
    assert np.abs(T - want).max() < 2e-3
    # the comparison separates a wrong permittivity: a stack of eps 2.0 misses by far more
    assert np.abs(transfer_matrix(stack(eps_hi=2.0), om) - T).max() > 0.02
