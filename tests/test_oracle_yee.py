"""Pins of the oracle's Yee + CPML field update (Eq. Maxwell, Yee's staggered grid).

Each check compares the oracle against something other than itself:
  * the discrete plane-wave eigenmode of the Yee scheme and its dispersion relation
    [sin(w dt/2)/dt]^2 = sum_a sin^2(k_a/2)  (closed form, exact to round-off);
  * the exact discrete energy invariant of leapfrog in a lossless closed box;
  * reflection from the CPML compared with a box large enough to have none.
"""
import numpy as np
import pytest

from paper_2512_06173_gb300.workloads import Problem


def eigenmode(shape, m, dt, t_e, e_dir):
    """Discrete Yee plane wave exp(i(k.r - w t)) sampled at the staggered positions."""
    nz, ny, nx = shape
    k = 2 * np.pi * np.array([m[0] / nx, m[1] / ny, m[2] / nz])
    K = 2 * np.sin(k / 2)
    E0 = np.cross(K, e_dir)
    E0 /= np.linalg.norm(E0)
    Om = np.linalg.norm(K)
    w = 2 / dt * np.arcsin(Om * dt / 2)
    H0 = np.cross(K, E0) / Om
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    off_E = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
    off_H = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]

    def wave(amp, off, t):
        ph = k[0] * (xx + off[0]) + k[1] * (yy + off[1]) + k[2] * (zz + off[2]) - w * t
        return amp * np.cos(ph)

    E = [wave(E0[a], off_E[a], t_e) for a in range(3)]
    H = [wave(H0[a], off_H[a], t_e - dt / 2) for a in range(3)]
    return E + H, w


@pytest.mark.parametrize("m,shape", [((1, 0, 0), (6, 5, 16)), ((1, 2, 1), (10, 12, 14)),
                                     ((0, 3, 2), (9, 16, 4))])
def test_plane_wave_dispersion(oracle_mod, m, shape):
    nz, ny, nx = shape
    dt = 0.5
    prob = Problem(nx, ny, nz, dt, periodic=(True, True, True))
    sim = oracle_mod.OracleSim(prob)
    f0, w = eigenmode(shape, m, dt, 0.0, np.array([0.3, -0.7, 0.5]))
    sim.set_fields(f0)
    nsteps = 300
    sim.step(nsteps)
    f1, _ = eigenmode(shape, m, dt, nsteps * dt, np.array([0.3, -0.7, 0.5]))
    got = sim.fields()
    err = max(np.abs(g - e).max() for g, e in zip(got, f1))
    assert err < 1e-10, err


def test_plane_wave_direction_and_speed(oracle_mod):
    """A pulse built from the +x eigenmode moves towards +x: a field started at
    H(t=-dt/2) of the backward wave would not match (guards the sign of the curls)."""
    shape = (4, 4, 32)
    dt = 0.5
    prob = Problem(32, 4, 4, dt, periodic=(True, True, True))
    sim = oracle_mod.OracleSim(prob)
    f0, w = eigenmode(shape, (1, 0, 0), dt, 0.0, np.array([0, 0, 1.0]))
    # backward wave: flip H
    fb = f0[:3] + [-h for h in f0[3:]]
    sim.set_fields(fb)
    sim.step(40)
    f1, _ = eigenmode(shape, (1, 0, 0), dt, 40 * dt, np.array([0, 0, 1.0]))
    err = max(np.abs(g - e).max() for g, e in zip(sim.fields(), f1))
    assert err > 0.1


def energy(eps, E, Hm, Hp):
    return 0.5 * sum((eps * e * e).sum() for e in E) + 0.5 * sum((a * b).sum() for a, b in zip(Hm, Hp))


def test_pec_box_energy_invariant(oracle_mod, W):
    """Lossless closed box with a random permittivity map: the leapfrog invariant
    W^n = 1/2 sum eps |E^n|^2 + 1/2 sum H^{n-1/2} . H^{n+1/2} is exact."""
    nx, ny, nz = 11, 9, 13
    rng = np.random.Generator(np.random.PCG64(7))
    mat = rng.integers(0, 3, size=(nz, ny, nx)).astype(np.uint8)
    materials = [W.Material(1.0), W.Material(2.25), W.Material(3.5)]
    prob = Problem(nx, ny, nz, 0.5, mat=mat, materials=materials)
    eps = np.array([m.eps_inf for m in materials])[mat]
    sim = oracle_mod.OracleSim(prob)
    f = W.random_fields(prob, 11)
    # PEC: tangential E on the index-0 walls is zero
    f[0][:, 0, :] = 0; f[0][0, :, :] = 0
    f[1][:, :, 0] = 0; f[1][0, :, :] = 0
    f[2][:, :, 0] = 0; f[2][:, 0, :] = 0
    sim.set_fields(f)
    E0, Hm0 = f[:3], f[3:]
    sim.step(1)
    Hp0 = sim.fields()[3:]
    W0 = energy(eps, E0, Hm0, Hp0)
    sim.step(1998)
    g = sim.fields()
    sim.step(1)
    Hp = sim.fields()[3:]
    W1 = energy(eps, g[:3], g[3:], Hp)
    assert abs(W1 - W0) / abs(W0) < 1e-12, (W0, W1)


def test_periodic_energy_invariant_mixed(oracle_mod, W):
    """Same invariant with two periodic axes and one walled axis."""
    nx, ny, nz = 8, 7, 10
    prob = Problem(nx, ny, nz, 0.5, periodic=(True, False, True))
    sim = oracle_mod.OracleSim(prob)
    f = W.random_fields(prob, 3)
    f[0][:, 0, :] = 0
    f[2][:, 0, :] = 0
    sim.set_fields(f)
    E0, Hm0 = f[:3], f[3:]
    sim.step(1)
    W0 = energy(1.0, E0, Hm0, sim.fields()[3:])
    sim.step(500)
    g = sim.fields()
    sim.step(1)
    W1 = energy(1.0, g[:3], g[3:], sim.fields()[3:])
    assert abs(W1 - W0) / abs(W0) < 1e-12


def blob(shape, c, w=1.5):
    nz, ny, nx = shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.exp(-((xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz + 0.5 - c[2]) ** 2) / (2 * w * w))


def test_cpml_reflection(oracle_mod):
    """A pulse leaving a 36^3 box through a 10-cell CPML matches, in the box interior,
    the same pulse in a 96^3 box whose walls are too far for any echo to return."""
    n, d, big = 36, 10, 96
    steps = 100  # t = 50: echoes from the small box's walls are back in the interior
    small = Problem(n, n, n, 0.5, pml=(d,) * 6)
    ref = Problem(big, big, big, 0.5)
    s1 = oracle_mod.OracleSim(small)
    s2 = oracle_mod.OracleSim(ref)
    z1 = [np.zeros((n, n, n))] * 6
    z2 = [np.zeros((big, big, big))] * 6
    c1 = (n / 2, n / 2, n / 2)
    c2 = (big / 2, big / 2, big / 2)
    f1 = list(z1); f1[2] = blob((n, n, n), c1)
    f2 = list(z2); f2[2] = blob((big, big, big), c2)
    s1.set_fields(f1); s2.set_fields(f2)
    # peak of the outgoing pulse as it crosses into the layer (t ~ 8)
    s1.step(16); s2.step(16)
    o = (big - n) // 2
    inc = np.abs(s2.fields()[2][o + d:o + n - d, o + d:o + n - d, o + d:o + n - d]).max()
    s1.step(steps - 16); s2.step(steps - 16)
    a = s1.fields()[2][d:n - d, d:n - d, d:n - d]
    b = s2.fields()[2][o + d:o + n - d, o + d:o + n - d, o + d:o + n - d]
    refl = np.abs(a - b).max() / inc
    assert refl < 1e-3, refl
    # without the layer the same box reflects at order one
    s3 = oracle_mod.OracleSim(Problem(n, n, n, 0.5))
    s3.set_fields(f1)
    s3.step(steps)
    refl0 = np.abs(s3.fields()[2][d:n - d, d:n - d, d:n - d] - b).max() / inc
    assert refl0 > 50 * refl


def test_cpml_profile_values(oracle_mod):
    """CPML coefficients follow the Roden-Gedney recursion b = exp(-(s/k + a) dt),
    c = s (b - 1) / (s k + k^2 a) with polynomial grading (Taflove & Hagness Ch. 7),
    evaluated here independently at a few depths."""
    prob = Problem(30, 4, 4, 0.5, periodic=(False, True, True), pml=(6, 8, 0, 0, 0, 0),
                   pml_kappa_max=3.0)
    sim = oracle_mod.OracleSim(prob)
    t = sim.pml_tables(0)
    m, smax, kmax, amax, dt = 3.0, 3.2, 3.0, 0.05, 0.5

    def ref(x):
        if x < 6:
            u = (6 - x) / 6
        elif x > 30 - 8:
            u = (x - 22) / 8
        else:
            return 0.0, 0.0, 1.0
        s = smax * u ** m
        k = 1 + (kmax - 1) * u ** m
        a = amax * (1 - u)
        b = np.exp(-(s / k + a) * dt)
        c = s * (b - 1) / (s * k + k * k * a) if s > 0 else 0.0
        return b, c, 1 / k

    for i in [0, 3, 5, 6, 15, 22, 23, 29]:
        b, c, ik = ref(float(i))
        assert np.allclose(t[0:3, i], [b, c, ik], rtol=1e-14, atol=0)
        b, c, ik = ref(i + 0.5)
        assert np.allclose(t[3:6, i], [b, c, ik], rtol=1e-14, atol=0)
