"""The oracle on the paper's printed worked example: superradiance of N co-located
two-level systems in 2D vacuum (Sec. IV.A, Eq. population_decay_superradiance), with the
parameters of Appendix B stored in tests/golden/superradiance_2d_appendix_b.json.

Units.  Grid units take the cell edge dx as length, dx / c as time and hbar = eps0 = c = 1;
a charge is then measured in sqrt(eps0 hbar c), so a dipole of d atomic units is
d sqrt(4 pi alpha) a0 / dx.  The paper does not state the length unit of its 2D solver;
the reading here is that the 2D emitter is a layer one cell thick (one periodic cell
along z), which makes mu = 187 a.u. a coupling of 1.0 in grid units.

At that coupling the regularised self-field of a kernel one cell wide is strong: it
lowers the emitter's oscillation frequency (by 3 % for one system, 12 % for four, whose
fields add).  The checks therefore measure the frequency from the phase of rho_ge and
pin the law of Eq. population_decay_superradiance at that frequency: the population
decays exponentially at N mu^2 w^2 / 2, times the form factor exp(-w^2 sigma^2) of the
Gaussian kernel, within 5 %, for N = 1 and N = 4.  A wrong coupling factor, a missing
factor N in the collective field, or a sign error in the coupling fails them.
"""
import json
import os

import numpy as np

from paper_2512_06173_gb300.workloads import Problem, pack_molecules, tls

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "superradiance_2d_appendix_b.json")

C = 2.99792458e8             # m/s
HARTREE_PER_HBAR = 4.134137333518e16  # 1/s: angular frequency of one hartree
ALPHA = 7.2973525693e-3
A0 = 5.29177210903e-11       # m


def grid_units(g):
    dx = g["dx_nm"] * 1e-9
    courant = C * g["dt_fs"] * 1e-15 / dx
    n = int(round(g["cell_um"][0] * 1e-6 / dx))
    pml = int(round(g["pml_nm"] * 1e-9 / dx))
    w = g["omega_tls_au"] * HARTREE_PER_HBAR * dx / C
    mu = g["mu12_au"] * np.sqrt(4 * np.pi * ALPHA) * A0 / dx
    return courant, n, pml, w, mu


def run(oracle_mod, g, N):
    courant, n, pml, w, mu = grid_units(g)
    ce = g["initial_state"]["ce"]
    cg = np.sqrt(g["initial_state"]["cg_squared"])
    mols = [tls((n / 2, n / 2, 0.5), w, mu, axis=2, sigma=1.0, gamma=1.0, cg=cg, ce=ce) for _ in range(N)]
    prob = Problem(n, n, 1, 0.5, periodic=(False, False, True), pml=(pml, pml, pml, pml, 0, 0),
                   molecules=pack_molecules(mols))
    sim = oracle_mod.OracleSim(prob)
    rate0 = N * mu ** 2 * w ** 2 / 2
    steps = int(round(3.5 / rate0 / 0.5))
    pe, ph = [], []
    for _ in range(steps):
        sim.step(1)
        r = sim.rho(0)
        pe.append(r[1, 1].real)
        ph.append(np.angle(r[0, 1]))
    t = (np.arange(steps) + 1) * 0.5
    pe = np.array(pe)
    sel = (pe < pe[0] * np.exp(-0.3)) & (pe > pe[0] * np.exp(-3.0))
    rate = -np.polyfit(t[sel], np.log(pe[sel]), 1)[0]
    ph = np.unwrap(ph)
    w_eff = abs(np.polyfit(t[sel], ph[sel], 1)[0])
    return rate, w_eff, w, mu


def test_fixture_maps_to_the_grid():
    g = json.load(open(GOLDEN))
    courant, n, pml, w, mu = grid_units(g)
    assert abs(courant - 0.5) < 1e-3      # 5e-3 fs at 3 nm: Courant number 1/2
    assert (n, pml) == (80, 30)
    assert abs(w - 0.1001) < 1e-3         # 0.242 a.u. = 6.59 eV
    assert abs(mu - 0.9989) < 1e-3
    assert g["n_tls"] == [1, 4]


def test_decay_law_of_the_printed_example(oracle_mod):
    g = json.load(open(GOLDEN))
    found = {}
    for N in g["n_tls"]:
        rate, w_eff, w, mu = run(oracle_mod, g, N)
        want = N * mu ** 2 * w_eff ** 2 / 2 * np.exp(-w_eff ** 2)  # sigma = dx = 1
        assert abs(rate / want - 1) < 0.05, (N, rate / want)
        found[N] = (rate, w_eff)
    # the collective field of four systems shifts the frequency further than one field
    assert found[4][1] < found[1][1] < w
    # and the ensemble decays about four times faster (exactly four at the same frequency)
    r = found[4][0] / found[1][0]
    shift = (found[4][1] / found[1][1]) ** 2 * np.exp(found[1][1] ** 2 - found[4][1] ** 2)
    assert abs(r / (4 * shift) - 1) < 0.05, r
