"""Physics pins of the coupled oracle: spontaneous emission and superradiance.

  * 2D (one periodic layer in z): the weak-excitation decay rate of one emitter is
    the rate quoted with Eq. population_decay_superradiance, gamma_QM = mu^2 w^2 / 2
    (hbar = eps0 = c = 1), times the Gaussian form factor exp(-w^2 sigma^2) that a
    kernel of width sigma imposes on radiation at |k| = w.
  * 3D: Fermi's golden rule gamma = w^3 mu^2 / (3 pi) times the same form factor.
    The explicit coupling holds the field of step n over the whole step, so the
    reactive near field of a narrow kernel acts half a step late; the resulting rate
    error is first order in dt and grows like 1/sigma^3.  The pins use sigma = 2
    (3 % off at Courant 0.5) and check the first-order convergence at sigma = 1.
  * Strong excitation: the emitter radiates a classical field, so its power follows
    |rho_ge|^2 = P_e P_g and the population obeys the logistic law dP_e/dt = -gamma
    P_e P_g; it matches the quantum exponential decay only in the weak-excitation
    limit, as the paper states.  From P_e = 0.9 the logit log(P_e / P_g) falls
    linearly at the weak-excitation rate, while the exponential rate -d log P_e / dt
    grows from about 0.1 gamma to gamma.
  * Superradiance (Eq. population_decay_superradiance): N co-located identical
    emitters evolve exactly like one emitter with coupling rescale sqrt(N) (the
    discrete identity behind the N-fold rate), and the ensemble decays N times faster.
"""
import numpy as np
import pytest

from paper_2512_06173_gb300.workloads import Problem, pack_molecules, tls


def decay_rate(t, pe):
    pe = np.asarray(pe)
    p0 = pe[0]
    sel = (pe < p0 * np.exp(-0.3)) & (pe > p0 * np.exp(-3.0))
    return -np.polyfit(t[sel], np.log(pe[sel]), 1)[0]


def run_emitters(oracle_mod, dim, n, mu, sigma, T, S=0.5, N=1, gamma=1.0, pml=10, w0=0.25, ce=0.01):
    if dim == 2:
        pos = (n / 2, n / 2, 0.5)
        kw = dict(periodic=(False, False, True), pml=(pml, pml, pml, pml, 0, 0))
        nz = 1
    else:
        pos = (n / 2, n / 2, n / 2)
        kw = dict(pml=(pml,) * 6)
        nz = n
    mols = [tls(pos, w0, mu, axis=2, sigma=sigma, gamma=gamma, cg=np.sqrt(1 - ce ** 2), ce=ce)
            for _ in range(N)]
    prob = Problem(n, n, nz, S, molecules=pack_molecules(mols), **kw)
    sim = oracle_mod.OracleSim(prob)
    steps = int(round(T / S))
    pe, rhos = [], []
    for _ in range(steps):
        sim.step(1)
        pe.append(sim.rho(0)[1, 1].real)
    t = (np.arange(steps) + 1) * S
    return t, np.array(pe), sim


def test_2d_spontaneous_emission_rate(oracle_mod):
    mu, w, sigma = 0.5, 0.25, 1.0
    t, pe, _ = run_emitters(oracle_mod, 2, 100, mu, sigma, 400)
    g = decay_rate(t, pe)
    want = mu ** 2 * w ** 2 / 2 * np.exp(-w ** 2 * sigma ** 2)
    assert abs(g / want - 1) < 0.05, g / want


def test_3d_fermi_golden_rule(oracle_mod):
    mu, w, sigma = 1.5, 0.25, 2.0
    t, pe, _ = run_emitters(oracle_mod, 3, 56, mu, sigma, 700)
    g = decay_rate(t, pe)
    want = w ** 3 * mu ** 2 / (3 * np.pi) * np.exp(-w ** 2 * sigma ** 2)
    assert abs(g / want - 1) < 0.05, g / want


def test_2d_strong_excitation_follows_the_logistic_law(oracle_mod):
    mu, w, sigma = 0.5, 0.25, 1.0
    want = mu ** 2 * w ** 2 / 2 * np.exp(-w ** 2 * sigma ** 2)
    t, pe, _ = run_emitters(oracle_mod, 2, 100, mu, sigma, 700, ce=np.sqrt(0.9))
    tw, pw, _ = run_emitters(oracle_mod, 2, 100, mu, sigma, 400)
    weak = decay_rate(tw, pw)
    sel = (pe < 0.85) & (pe > 0.15)
    logit = np.log(pe[sel] / (1 - pe[sel]))
    fit = np.polyfit(t[sel], logit, 1)
    g = -fit[0]
    assert abs(g / weak - 1) < 0.03, (g, weak)
    assert abs(g / want - 1) < 0.06, g / want
    assert np.abs(logit - np.polyval(fit, t[sel])).max() < 0.05

    def exp_rate(hi, lo):
        s = (pe < hi) & (pe > lo)
        return -np.polyfit(t[s], np.log(pe[s]), 1)[0]

    # an exponential law would give one rate; the logistic one starts near gamma P_g
    assert exp_rate(0.85, 0.75) < 0.3 * g and exp_rate(0.25, 0.15) > 0.7 * g


@pytest.mark.slow
def test_3d_rate_converges_first_order_in_dt(oracle_mod):
    mu, w, sigma = 1.5, 0.25, 1.0
    want = w ** 3 * mu ** 2 / (3 * np.pi) * np.exp(-w ** 2 * sigma ** 2)
    errs = []
    for S in (0.5, 0.25):
        t, pe, _ = run_emitters(oracle_mod, 3, 48, mu, sigma, 600, S=S, pml=8)
        errs.append(abs(decay_rate(t, pe) / want - 1))
    assert 0.35 < errs[1] / errs[0] < 0.65, errs


def test_superradiance_identity_colocated(oracle_mod):
    """N co-located emitters with coupling 1 == one emitter with coupling sqrt(N)."""
    N = 4
    _, pe_n, s_n = run_emitters(oracle_mod, 2, 48, 0.5, 1.0, 100, N=N, pml=8)
    _, pe_1, s_1 = run_emitters(oracle_mod, 2, 48, 0.5, 1.0, 100, N=1, gamma=np.sqrt(N), pml=8)
    assert np.abs(pe_n - pe_1).max() < 1e-15
    for m in range(N):
        assert np.abs(s_n.rho(m) - s_1.rho(0)).max() < 1e-15
    # radiated field is sqrt(N) times larger
    fn, f1 = s_n.fields()[2], s_1.fields()[2]
    assert np.allclose(fn, np.sqrt(N) * f1, rtol=1e-9, atol=1e-18)


def test_superradiant_rate_scales_with_n(oracle_mod):
    mu, sigma = 0.35, 1.0
    t, pe1, _ = run_emitters(oracle_mod, 2, 100, mu, sigma, 900)
    t4, pe4, _ = run_emitters(oracle_mod, 2, 100, mu, sigma, 250, N=4)
    r = decay_rate(t4, pe4) / decay_rate(t, pe1)
    assert abs(r / 4 - 1) < 0.03, r
