"""Pins of the oracle on the resonance-energy-transfer workload (Sec. IV.B setup, with
model acceptors): a two-level donor in a coherent state radiating onto a ground-state
acceptor in 3D vacuum.

- embedding: an 8-level acceptor whose other six levels have no dipole to anything
  evolves, on its two coupled levels, exactly as the two-level acceptor of the same
  transition (same fields, same 2x2 block of rho), with a complex transition dipole so
  that a transposed operand anywhere in the multilevel step would show;
- weak coupling: the acceptor's energy gain is second order in the coupling, so it
  scales as mu_A^2 at a fixed donor and as mu_D^2 at a fixed acceptor while the donor
  stays far from decaying (ratios of 4 for doubled dipoles).
"""
import dataclasses

import numpy as np
import pytest

from paper_2512_06173_gb300 import workloads as W


def _acceptor_gain(oracle_mod, prob, steps):
    o = oracle_mod.OracleSim(prob)
    o.step(steps)
    H = prob.molecules.matrix(prob.molecules.H0, 1)
    return float(np.real(np.trace(o.rho(1) @ H)))


def test_uncoupled_levels_do_not_change_the_transfer(oracle_mod):
    base = W.energy_transfer(edge=32, distance=10, n_acceptor=2, pml=6)
    don = W.tls(tuple(base.molecules.pos[0]), 0.25, 2.0, axis=2, cg=np.sqrt(0.5), ce=np.sqrt(0.5))
    pos_a = tuple(base.molecules.pos[1])
    mu = 0.3 * np.exp(0.7j)  # strong acceptor so that the transfer is well above round-off
    w = 0.25
    # two-level acceptor, RK4 like the multilevel one
    mu2 = np.zeros((3, 2, 2), np.complex128)
    mu2[2] = [[0, mu], [np.conj(mu), 0]]
    rho2 = np.diag([1.0, 0.0]).astype(np.complex128)
    acc2 = dict(n=2, pos=pos_a, sigma=1.5, gamma=1.0, H0=np.diag([0.0, w]).astype(np.complex128), mu=mu2,
                rho=rho2, decay=0.0, dephase=0.0, kind=W.KIND_RK4, nsub=1)
    # the same transition between levels 0 and 3 of eight, the other levels at their own energies
    k = 3
    E = np.array([0.0, 0.16, 0.21, w, 0.31, 0.44, 0.52, 0.6])
    mu8 = np.zeros((3, 8, 8), np.complex128)
    mu8[2, 0, k], mu8[2, k, 0] = mu, np.conj(mu)
    rho8 = np.zeros((8, 8), np.complex128)
    rho8[0, 0] = 1.0
    acc8 = dict(acc2, n=8, H0=np.diag(E).astype(np.complex128), mu=mu8, rho=rho8)
    pa = base.replace(molecules=W.pack_molecules([don, acc2]))
    pb = base.replace(molecules=W.pack_molecules([don, acc8]))
    a, b = oracle_mod.OracleSim(pa), oracle_mod.OracleSim(pb)
    a.step(240)
    b.step(240)
    ra, rb = a.rho(1), b.rho(1)
    assert np.real(ra[1, 1]) > 1e-5  # energy has been transferred
    sel = [0, k]
    assert np.abs(rb[np.ix_(sel, sel)] - ra).max() < 1e-13
    rest = np.ones((8, 8), bool)
    rest[np.ix_(sel, sel)] = False
    assert np.abs(rb[rest]).max() == 0.0
    for x, y in zip(a.fields(), b.fields()):
        assert np.abs(x - y).max() < 1e-13 * max(np.abs(x).max(), 1e-30)


@pytest.mark.parametrize("which", ["acceptor", "donor"])
def test_gain_is_second_order_in_each_dipole(oracle_mod, which):
    if which == "acceptor":  # donor dipole 2 in both runs
        p1 = W.energy_transfer(edge=36, distance=10, pml=8, mu_acceptor=0.02, ratio=100.0)
        p2 = W.energy_transfer(edge=36, distance=10, pml=8, mu_acceptor=0.04, ratio=50.0)
    else:  # donor dipole 0.2 -> 0.4: decay over the run ~ 1e-2
        p1 = W.energy_transfer(edge=36, distance=10, pml=8, mu_acceptor=0.02, ratio=10.0)
        p2 = W.energy_transfer(edge=36, distance=10, pml=8, mu_acceptor=0.02, ratio=20.0)
    g1, g2 = _acceptor_gain(oracle_mod, p1, 300), _acceptor_gain(oracle_mod, p2, 300)
    assert g1 > 0
    assert abs(g2 / g1 - 4.0) < 2e-3


def test_workload_generators_are_seeded_and_well_formed():
    """The energy-transfer realisations repeat for a seed; each acceptor has a Hermitian
    z-dipole, sorted levels from 0, the donor-resonant level with the strongest ground
    dipole, and starts in the ground state; the donor starts in (1/sqrt 2, 1/sqrt 2)."""
    a = W.energy_transfer_batch(count=12, edge=48)
    b = W.energy_transfer_batch(count=12, edge=48)
    assert [p.name for p in a] == [p.name for p in b]
    assert {int(p.molecules.nlev[1]) for p in a} <= {2, 4, 8}
    for p, q in zip(a, b):
        m = p.molecules
        assert np.array_equal(m.pos, q.molecules.pos) and np.array_equal(m.mu, q.molecules.mu)
        assert np.array_equal(m.H0, q.molecules.H0)
        n = int(m.nlev[1])
        H = m.matrix(m.H0, 1)
        E = np.real(np.diag(H))
        assert E[0] == 0.0 and np.all(np.diff(E) >= 0)
        mz = m.matrix(m.mu[2], 1)
        assert np.allclose(mz, mz.conj().T, atol=0)
        assert np.all(m.matrix(m.mu[0], 1) == 0) and np.all(m.matrix(m.mu[1], 1) == 0)
        k = int(np.argmax(np.abs(mz[0])))
        assert E[k] == 0.25 and abs(mz[0, k]) == 0.02
        r = m.matrix(m.rho0, 1)
        assert r[0, 0] == 1.0 and np.abs(r).sum() == 1.0
        rd = m.matrix(m.rho0, 0)
        assert np.allclose(rd, 0.5) and m.kind[1] == W.KIND_RK4
        assert abs(m.pos[1, 0] - m.pos[0, 0] - float(p.name.split("-d")[1].split("-")[0])) < 1e-3
        assert n == len(E)
