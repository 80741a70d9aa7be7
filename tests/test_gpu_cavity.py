"""Single-mode cavity (ml_cavity_*) through the C ABI against the oracle's cavity
(oracle/cavity.py) on the same seeded molecules: the mode state (q, p, d of both
polarisations) after every step and the final density matrices.  FP64 agrees to
round-off (relative 1e-10 on the mode, 1e-9 on the density matrices), FP32 within
1e-4 (measured: 3.5e-6 on the mode, 1.8e-6 on the density matrices).  Also at 3,000 two-level emitters (the
two-level path and the multi-block dipole sum), the sqrt(N) identity on the GPU, and
refusal of bad descriptors.
"""
import numpy as np
import pytest

from paper_2512_06173_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ml():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2512_06173_gb300 import maxlink
    maxlink.load()
    return maxlink


@pytest.fixture(scope="module")
def cav():
    from oracle import cavity
    return cavity


def mixed(seed, M):
    """Exact two-level, two-level with dephasing (RK4) and 3..5-level ladders with decay,
    in-plane dipoles of random direction, seeded states."""
    rng = np.random.default_rng(seed)
    mats = []
    for m in range(M):
        kind = m % 3
        th = rng.uniform(0, 2 * np.pi)
        if kind < 2:
            ce = np.sqrt(rng.uniform(0, 0.3)) * np.exp(1j * rng.uniform(0, 2 * np.pi))
            d = W.tls((4.0, 4.0, 4.0), rng.uniform(0.22, 0.28), rng.uniform(0.5, 1.2), axis=0,
                      gamma=rng.uniform(0.5, 1.5), cg=np.sqrt(1 - abs(ce) ** 2), ce=ce,
                      dephase=0.0 if kind == 0 else 1e-3)
            mu = d["mu"][0].copy()
            d["mu"] = np.stack([np.cos(th) * mu, np.sin(th) * mu, 0 * mu])
        else:
            n = 3 + m % 3
            H0 = np.diag(np.cumsum([0.0] + list(0.25 * (1 + 0.05 * rng.standard_normal(n - 1))))).astype(complex)
            ladder = np.diag(np.sqrt(np.arange(1, n)), 1).astype(complex)
            x = 0.4 * (ladder + ladder.T)
            c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
            c[0] += 3.0
            c /= np.linalg.norm(c)
            d = dict(n=n, pos=(4.0, 4.0, 4.0), sigma=1.0, gamma=rng.uniform(0.5, 1.5), H0=H0,
                     mu=np.stack([np.cos(th) * x, np.sin(th) * x, 0 * x]), rho=np.outer(c, c.conj()),
                     decay=1e-3, dephase=0.0, kind=1, nsub=2)
        mats.append(d)
    return W.pack_molecules(mats)


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("precision,tol,rho_tol", [(1, 1e-10, 1e-9), (0, 1e-4, 1e-4)])
def test_matches_oracle_every_step(ml, cav, precision, tol, rho_tol):
    mols = mixed(0, 12)
    kw = dict(omega_c=0.25, coupling=0.01, dt=0.5, q0=(0.3, -0.2), p0=(0.0, 0.1))
    o = cav.OracleCavity(mols, **kw)
    g = ml.Cavity(mols, precision=precision, **kw)
    try:
        assert rel(g.mode(), o.mode()) < 1e-12  # the initial dipoles
        for _ in range(150):
            g.step(1)
            o.step(1)
            assert rel(g.mode(), o.mode()) < tol
        for m in range(mols.count):
            assert rel(g.rho(m), o.rho(m)) < rho_tol  # FP32 measured: 1.8e-6
        assert g.nstep == 150
    finally:
        g.close()


def test_three_thousand_two_level_emitters(ml, cav):
    rng = np.random.default_rng(5)
    M = 3000
    mats = [W.tls((4.0, 4.0, 4.0), 0.25, 0.05, axis=m % 2, gamma=1.0, cg=np.sqrt(1 - 1e-6),
                  ce=1e-3 * np.exp(1j * rng.uniform(0, 2 * np.pi))) for m in range(M)]
    mols = W.pack_molecules(mats)
    kw = dict(omega_c=0.25, coupling=0.002, dt=0.5)
    o = cav.OracleCavity(mols, **kw)
    g = ml.Cavity(mols, precision=1, **kw)
    try:
        for _ in range(25):
            g.step(1)
            o.step(1)
        assert rel(g.mode(), o.mode()) < 1e-10
        pops = g.molecules(ml.ML_MOL_POP)
        po = np.array([np.real(np.diag(o.rho(m))) for m in range(M)])
        assert np.abs(pops[:, :2] - po).max() < 1e-12
    finally:
        g.close()


def test_blocks_with_several_rows(ml, cav):
    """120,000 exact two-level emitters (the cavity workload's ensemble): more rows of 256
    than the one-launch kernel has blocks (456), so some blocks add two rows, and the last
    row is ragged (192 molecules).  Mode after every step and sampled density matrices
    against the oracle, FP64 and FP32."""
    M = 120_000
    mols = W.cavity_ensemble(M)
    eps = 0.05 * 0.25 ** 2 / np.sqrt(2 * 0.25 * M * 0.05 ** 2 / 2)
    kw = dict(omega_c=0.25, coupling=eps, dt=0.5, q0=(2e-3, -1e-3), p0=(0.0, 5e-4))
    o = cav.OracleCavity(mols, **kw)
    gs = {prec: ml.Cavity(mols, precision=prec, **kw) for prec in (1, 0)}
    tol = {1: 1e-10, 0: 1e-4}
    sample = np.r_[0:8, 255:259, 116_730:116_745, M - 200:M]
    try:
        for _ in range(4):
            o.step(1)
            for prec, g in gs.items():
                g.step(1)
                assert rel(g.mode(), o.mode()) < tol[prec], prec
        for prec, g in gs.items():
            pool = g.molecules(ml.ML_MOL_RHO)  # two levels each: molecule m at 4 m
            for m in sample:
                assert rel(pool[4 * m:4 * m + 4].reshape(2, 2), o.rho(int(m))) < tol[prec], (prec, m)
    finally:
        for g in gs.values():
            g.close()


def test_sqrt_n_identity(ml):
    N = 7
    kw = dict(omega0=0.25, mu12=0.8, axis=1, cg=np.sqrt(0.7), ce=np.sqrt(0.3) * np.exp(0.4j), dephase=1e-3)
    many = ml.Cavity(W.pack_molecules([W.tls((4.0, 4.0, 4.0), **kw) for _ in range(N)]), 0.25, 0.02, 0.5,
                     precision=1)
    one = ml.Cavity(W.pack_molecules([W.tls((4.0, 4.0, 4.0), gamma=np.sqrt(N), **kw)]), 0.25, 0.02, 0.5,
                    precision=1)
    try:
        many.step(400)
        one.step(400)
        a, b = many.mode(), one.mode()
        assert np.abs(a[:4] - np.sqrt(N) * b[:4]).max() < 1e-10 * max(1.0, np.abs(a).max())
        for m in range(N):
            assert np.abs(many.rho(m) - one.rho(0)).max() < 1e-12
    finally:
        many.close()
        one.close()


def test_refuses_bad_descriptors(ml):
    mols = mixed(1, 3)
    for kw in (dict(omega_c=0.0, coupling=0.01, dt=0.5), dict(omega_c=0.25, coupling=0.01, dt=-1.0),
               dict(omega_c=0.25, coupling=float("nan"), dt=0.5)):
        with pytest.raises(ml.MaxlinkError) as e:
            ml.Cavity(mols, **kw)
        assert e.value.status == ml.ML_ERR_INVALID_ARG
    with pytest.raises(ml.MaxlinkError):
        ml.Cavity(W.empty_molecules(), 0.25, 0.01, 0.5)


@pytest.mark.parametrize("two_level", [False, True])
def test_graph_replay_equals_single_steps(ml, two_level):
    """130 steps as two replays of the captured 64-step sequence plus two single steps
    give the bits of 130 separate calls (both molecule kernels)."""
    mols = (W.pack_molecules([W.tls((4.0, 4.0, 4.0), 0.25, 0.3, axis=m % 2, cg=np.sqrt(0.9), ce=np.sqrt(0.1),
                                    dephase=1e-3 * (m % 2)) for m in range(300)])
            if two_level else mixed(2, 30))
    a = ml.Cavity(mols, 0.25, 0.01, 0.5, q0=(0.2, 0.1))
    b = ml.Cavity(mols, 0.25, 0.01, 0.5, q0=(0.2, 0.1))
    try:
        for _ in range(130):
            a.step(1)
        b.step(130)
        assert np.array_equal(a.mode(), b.mode())
        assert np.array_equal(a.molecules(ml.ML_MOL_RHO), b.molecules(ml.ML_MOL_RHO))
        assert a.nstep == b.nstep == 130
    finally:
        a.close()
        b.close()
