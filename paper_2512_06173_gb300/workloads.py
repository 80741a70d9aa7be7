"""Seeded synthetic inputs for the coupled Yee/molecule step.

This module only *describes* problems: grid sizes, boundary layers, material maps,
sources, molecule tables and flux planes, drawn from numpy PCG64 generators with
fixed seeds.  It holds none of the method's arithmetic (no field update, no kernel
weights, no propagator); both the CUDA library binding and the FP64 oracle consume
the same `Problem` objects and each converts them on its own.

Units are grid units with c = eps0 = mu0 = hbar = 1 and a cell edge of 1 (the MEEP
convention the paper adopts in Appendix A), so the time step equals the Courant
number.

Workload shapes follow the paper's examples (Sec. IV and Appendix B):
superradiant emitter ensembles (Sec. IV.A), a Bragg resonator with a vibrational
ensemble (Sec. IV.C) and a metal nanostructure with a molecular shell (Sec. IV.D).
The paper's own inputs (MEEP geometries, water and HCN data) are not available, so
these synthetic problems stand in for them.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Propagator kinds for molecules.
KIND_EXACT2 = 0  # two-level, no dissipation: exact exponential of the held 2x2 Hamiltonian
KIND_RK4 = 1     # any level count 2..8, optional Lindblad terms: classic RK4 substeps

MAX_LEVELS = 8


@dataclass
class Source:
    """Soft current sheet on the plane index `index` normal to `axis`,
    polarised along `comp`, time profile amp*exp(-((t-t0)/width)^2/2)*cos(omega*(t-t0))."""
    axis: int
    index: int
    comp: int
    amp: float
    omega: float
    width: float
    t0: float


@dataclass
class FluxPlane:
    axis: int
    index: int
    omegas: np.ndarray  # float64 (nfreq,)


@dataclass
class Material:
    """eps_inf plus dispersive poles, each dJ/dt + gamma J + omega0^2 P = wp^2 E with
    dP/dt = J, their currents summed: omega0 = 0 is a Drude term (wp the plasma
    frequency), omega0 > 0 a Lorentz oscillator (wp^2 = delta_eps omega0^2).  The first
    pole is (wp, gamma, omega0); `extra` holds up to MAX_POLES - 1 more."""
    eps_inf: float = 1.0
    wp: float = 0.0      # pole strength (0: no pole)
    gamma: float = 0.0   # pole damping
    omega0: float = 0.0  # pole resonance (0: Drude)
    extra: Tuple[Tuple[float, float, float], ...] = ()  # further poles (wp, gamma, omega0)

    def poles(self) -> List[Tuple[float, float, float]]:
        """The material's poles with wp > 0, in order: the first, then `extra`."""
        ps = [(self.wp, self.gamma, self.omega0)] + [tuple(map(float, p)) for p in self.extra]
        return [p for p in ps if p[0] > 0]


MAX_POLES = 4  # dispersive poles per material


@dataclass
class Molecules:
    """Packed molecule table.  Matrices of molecule m live at pool[off[m] : off[m]+n*n]
    (row-major n x n, complex128)."""
    nlev: np.ndarray      # int32 (M,)
    off: np.ndarray       # int64 (M,)
    pos: np.ndarray       # float64 (M,3), grid units, cell (i,j,k) spans [i,i+1) x ...
    sigma: np.ndarray     # float64 (M,) Gaussian width in cells
    gamma: np.ndarray     # float64 (M,) coupling rescale (Eq. Polarization_mol)
    decay: np.ndarray     # float64 (M,) ladder decay rate (Lindblad, k -> k-1)
    dephase: np.ndarray   # float64 (M,) pure dephasing rate of every coherence
    kind: np.ndarray      # int32 (M,) KIND_EXACT2 | KIND_RK4
    nsub: np.ndarray      # int32 (M,) RK4 substeps per field step
    H0: np.ndarray        # complex128 pool
    mu: np.ndarray        # complex128 (3, pool) dipole operators x, y, z
    rho0: np.ndarray      # complex128 pool, initial density matrices

    @property
    def count(self) -> int:
        return int(self.nlev.shape[0])

    def matrix(self, pool: np.ndarray, m: int) -> np.ndarray:
        n = int(self.nlev[m])
        o = int(self.off[m])
        return pool[o:o + n * n].reshape(n, n)

    def subset(self, idx: Sequence[int]) -> "Molecules":
        idx = np.asarray(idx, dtype=np.int64)
        nl = self.nlev[idx]
        sizes = nl.astype(np.int64) ** 2
        off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        total = int(sizes.sum())
        H0 = np.zeros(total, np.complex128)
        mu = np.zeros((3, total), np.complex128)
        rho = np.zeros(total, np.complex128)
        for new, old in enumerate(idx):
            s = int(sizes[new])
            o, oo = int(off[new]), int(self.off[old])
            H0[o:o + s] = self.H0[oo:oo + s]
            mu[:, o:o + s] = self.mu[:, oo:oo + s]
            rho[o:o + s] = self.rho0[oo:oo + s]
        return Molecules(nl.copy(), off, self.pos[idx].copy(), self.sigma[idx].copy(),
                         self.gamma[idx].copy(), self.decay[idx].copy(),
                         self.dephase[idx].copy(), self.kind[idx].copy(),
                         self.nsub[idx].copy(), H0, mu, rho)


def empty_molecules() -> Molecules:
    z = np.zeros(0)
    return Molecules(np.zeros(0, np.int32), np.zeros(0, np.int64), np.zeros((0, 3)), z.copy(),
                     z.copy(), z.copy(), z.copy(), np.zeros(0, np.int32), np.zeros(0, np.int32),
                     np.zeros(0, np.complex128), np.zeros((3, 0), np.complex128),
                     np.zeros(0, np.complex128))


def pack_molecules(mats: List[dict]) -> Molecules:
    """Pack a list of per-molecule dicts with keys n, pos, sigma, gamma, H0 (n x n),
    mu (3, n, n), rho (n x n) and optional decay, dephase, kind, nsub."""
    M = len(mats)
    nlev = np.array([d["n"] for d in mats], np.int32)
    sizes = nlev.astype(np.int64) ** 2
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64) if M else np.zeros(0, np.int64)
    total = int(sizes.sum())
    H0 = np.zeros(total, np.complex128)
    mu = np.zeros((3, total), np.complex128)
    rho = np.zeros(total, np.complex128)
    for m, d in enumerate(mats):
        o, s = int(off[m]), int(sizes[m])
        H0[o:o + s] = np.asarray(d["H0"], np.complex128).ravel()
        mu[:, o:o + s] = np.asarray(d["mu"], np.complex128).reshape(3, s)
        rho[o:o + s] = np.asarray(d["rho"], np.complex128).ravel()
    decay = np.array([d.get("decay", 0.0) for d in mats], np.float64)
    deph = np.array([d.get("dephase", 0.0) for d in mats], np.float64)
    kind = np.array([d.get("kind", KIND_EXACT2 if (d["n"] == 2 and d.get("decay", 0.0) == 0.0
                                                   and d.get("dephase", 0.0) == 0.0) else KIND_RK4)
                     for d in mats], np.int32)
    nsub = np.array([d.get("nsub", 1) for d in mats], np.int32)
    pos = np.array([d["pos"] for d in mats], np.float64).reshape(M, 3)
    sigma = np.array([d["sigma"] for d in mats], np.float64)
    gamma = np.array([d.get("gamma", 1.0) for d in mats], np.float64)
    return Molecules(nlev, off, pos, sigma, gamma, decay, deph, kind, nsub, H0, mu, rho)


def tls(pos, omega0, mu12, axis=2, sigma=1.5, gamma=1.0, cg=1.0, ce=0.0, dephase=0.0,
        decay=0.0, kind=None, nsub=1) -> dict:
    """Two-level emitter: H0 = diag(0, omega0), mu = mu12 * e_axis * sigma_x (Eq. von-Neumann-tls)."""
    H0 = np.diag([0.0, omega0]).astype(np.complex128)
    mu = np.zeros((3, 2, 2), np.complex128)
    mu[axis] = mu12 * np.array([[0, 1], [1, 0]])
    c = np.array([cg, ce], np.complex128)
    rho = np.outer(c, c.conj())
    d = dict(n=2, pos=pos, sigma=sigma, gamma=gamma, H0=H0, mu=mu, rho=rho,
             dephase=dephase, decay=decay, nsub=nsub)
    if kind is not None:
        d["kind"] = kind
    return d


@dataclass
class Problem:
    nx: int
    ny: int
    nz: int
    courant: float = 0.5
    periodic: Tuple[bool, bool, bool] = (False, False, False)
    pml: Tuple[int, int, int, int, int, int] = (0, 0, 0, 0, 0, 0)
    pml_m: float = 3.0
    pml_sigma_max: float = 3.2        # 0.8 (m+1) / (eta dx) with eta = dx = 1
    pml_kappa_max: float = 1.0
    pml_alpha_max: float = 0.05
    mat: Optional[np.ndarray] = None  # uint8 (nz, ny, nx) material index
    materials: List[Material] = field(default_factory=lambda: [Material()])
    design_box: Optional[Tuple[int, int, int, int, int, int]] = None  # x0,y0,z0,sx,sy,sz
    design_eps: Optional[np.ndarray] = None  # float64 (sz, sy, sx) relative permittivity
    sources: List[Source] = field(default_factory=list)
    molecules: Molecules = field(default_factory=empty_molecules)
    planes: List[FluxPlane] = field(default_factory=list)
    name: str = "custom"
    zchunk: int = 0  # planes per z chunk of the field pass (0: automatic; see ml_grid_desc)

    @property
    def dt(self) -> float:
        return float(self.courant)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------------
# Workloads shaped like the paper's examples.
# ----------------------------------------------------------------------------------

def plain_single_emitter(dtype_note: str = "") -> Problem:
    """40^3 cells, Courant 0.5, vacuum, 8-cell CPML on all faces, one two-level
    emitter at the grid centre (omega0 = 0.25, mu12 = 0.1 along z, sigma = 2 cells),
    initial amplitudes (sqrt(0.9), sqrt(0.1)), no Lindblad terms."""
    n = 40
    mol = pack_molecules([tls((n / 2, n / 2, n / 2), 0.25, 0.1, axis=2, sigma=2.0,
                              cg=np.sqrt(0.9), ce=np.sqrt(0.1))])
    return Problem(n, n, n, 0.5, pml=(8,) * 6, molecules=mol, name="plain-40^3-1tls")


def superradiant_slab(n: int = 256, nmol: int = 10000, slab: int = 32, pml: int = 10,
                      nfreq: int = 8, seed: int = 2) -> Problem:
    """Vacuum cube with `nmol` two-level emitters (omega0 = 0.25, mu12 = 0.02 along z,
    sigma = 1.5 cells) at seeded uniform positions in a `slab`-cell-thick central slab,
    all excited with a seeded random coherence of 1e-3 and pure dephasing 1e-5; flux
    planes on both sides at `nfreq` frequencies in [0.20, 0.30].  Stand-in for the
    superradiance example of Sec. IV.A at 3D scale."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = pml + 2, n - pml - 2
    zc = n // 2
    xs = rng.uniform(lo, hi, size=nmol)
    ys = rng.uniform(lo, hi, size=nmol)
    zs = rng.uniform(zc - slab // 2, zc + slab // 2, size=nmol)
    phi = rng.uniform(0.0, 2 * np.pi, size=nmol)
    mats = []
    for m in range(nmol):
        cg = 1e-3 * np.exp(1j * phi[m])
        ce = np.sqrt(1.0 - 1e-6)
        mats.append(tls((xs[m], ys[m], zs[m]), 0.25, 0.02, axis=2, sigma=1.5,
                        cg=cg, ce=ce, dephase=1e-5))
    om = np.linspace(0.20, 0.30, nfreq)
    planes = [FluxPlane(2, pml + 4, om.copy()), FluxPlane(2, n - pml - 4, om.copy())]
    return Problem(n, n, n, 0.5, pml=(pml,) * 6, molecules=pack_molecules(mats),
                   planes=planes, name=f"superradiant-slab-{n}^3-{nmol}tls")


def dispersive_stack(nx: int = 512, ny: int = 512, nz: int = 256, nmol: int = 20000, pml: int = 10,
                     layer: int = 32, film: int = 8, nfreq: int = 8, seed: int = 5, width: float = 20.0,
                     t0: float = 80.0) -> Problem:
    """Planar dispersive stack, periodic in x and y with CPML on the z faces: a
    `layer`-cell Lorentz dielectric (eps_inf 1.5, delta_eps 1, omega0 0.3, gamma 0.01)
    centred in z on a `film`-cell Drude-Lorentz metal film (Drude wp 1, gamma 0.05 plus
    an interband Lorentz pole wp 0.5, omega0 0.6, gamma 0.1) that mirrors the pulse; `nmol` ground-state two-level emitters (omega0 = 0.25, mu12 = 0.05 along x,
    sigma = 1.5 cells) at seeded uniform positions in the middle of the Lorentz layer;
    an x-polarised Gaussian-pulse current sheet (omega 0.25, temporal `width`, centred at
    `t0`) near the lower CPML and
    flux planes on both sides.  Stand-in for the emitters in dispersive media
    (Drude/Lorentz dielectric functions) that the grid solver of Sec. II.A supports."""
    rng = np.random.Generator(np.random.PCG64(seed))
    zc = nz // 2
    mat = np.zeros((nz, ny, nx), np.uint8)
    mat[zc - layer // 2:zc + layer // 2] = 1
    mat[zc + layer // 2:zc + layer // 2 + film] = 2
    materials = [Material(1.0), Material(1.5, wp=0.3, gamma=0.01, omega0=0.3), Material(1.0, wp=1.0, gamma=0.05, extra=((0.5, 0.1, 0.6),))]
    xs = rng.uniform(0, nx, size=nmol)
    ys = rng.uniform(0, ny, size=nmol)
    zs = rng.uniform(zc - layer // 4, zc + layer // 4, size=nmol)
    mols = [tls((xs[m], ys[m], zs[m]), 0.25, 0.05, axis=0, sigma=1.5) for m in range(nmol)]
    om = np.linspace(0.20, 0.30, nfreq)
    planes = [FluxPlane(2, pml + 6, om.copy()), FluxPlane(2, nz - pml - 4, om.copy())]
    src = [Source(axis=2, index=pml + 2, comp=0, amp=1.0, omega=0.25, width=width, t0=t0)]
    return Problem(nx, ny, nz, 0.5, periodic=(True, True, False), pml=(0, 0, 0, 0, pml, pml), mat=mat,
                   materials=materials, sources=src, molecules=pack_molecules(mols), planes=planes,
                   name=f"dispersive-stack-{nx}x{ny}x{nz}-{nmol}tls")


def random_hermitian(rng, n, std):
    a = rng.normal(0, std, (n, n)) + 1j * rng.normal(0, std, (n, n))
    return (a + a.conj().T) / 2


def bragg_ensemble(nx=512, ny=512, nz=384, nmol=100000, pml=10, slab=32, seed=3,
                   layers=12, nfreq=8, width=20.0) -> Problem:
    """Bragg-mirror stack (alternating eps 2.25 / 1.0 quarter-wave layers at omega =
    0.25, 4 and 6 cells) along x, split around a central `slab`-cell slab holding
    `nmol` multilevel systems with level count uniform in 2..8, Hermitian z-dipoles
    with N(0, 0.01) entries, harmonic ladders with spacing 0.2 +- 5 % and log-uniform
    decay rates in [1e-6, 1e-4]; a z-polarised Gaussian-pulse current sheet on the
    plane x = pml + 2 and flux planes on both sides.  The pulse travels along x, so the
    z-polarised field and the z-dipoles couple.  Stand-in for the Bragg resonator of
    Sec. IV.C."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mat = np.zeros((nz, ny, nx), np.uint8)
    xc = nx // 2
    half = layers // 2
    # stack on both sides of the slab: (4 cells eps 2.25, 6 cells eps 1) x half
    # (on a grid too narrow for the whole stack the layers that would leave it are dropped)
    x = xc + slab // 2
    for _ in range(half):
        if x + 4 <= nx:
            mat[:, :, x:x + 4] = 1
        x += 10
    x = xc - slab // 2
    for _ in range(half):
        if x - 4 >= 0:
            mat[:, :, x - 4:x] = 1
        x -= 10
    mats = []
    nl = rng.integers(2, 9, size=nmol)
    px = rng.uniform(xc - slab // 2, xc + slab // 2, size=nmol)
    py = rng.uniform(pml + 7, ny - pml - 7, size=nmol)
    pz = rng.uniform(pml + 7, nz - pml - 7, size=nmol)
    rates = np.exp(rng.uniform(np.log(1e-6), np.log(1e-4), size=nmol))
    for m in range(nmol):
        n = int(nl[m])
        steps = 0.2 * (1 + rng.uniform(-0.05, 0.05, size=n - 1))
        E = np.concatenate([[0.0], np.cumsum(steps)])
        mu = np.zeros((3, n, n), np.complex128)
        mu[2] = random_hermitian(rng, n, 0.01)
        rho = np.zeros((n, n), np.complex128)
        rho[0, 0] = 1.0
        mats.append(dict(n=n, pos=(px[m], py[m], pz[m]), sigma=1.5, gamma=1.0,
                         H0=np.diag(E).astype(np.complex128), mu=mu, rho=rho,
                         decay=float(rates[m]), kind=KIND_RK4, nsub=1))
    src = [Source(axis=0, index=pml + 2, comp=2, amp=1.0, omega=0.25, width=width, t0=5.0 * width)]
    om = np.linspace(0.20, 0.30, nfreq)
    planes = [FluxPlane(0, pml + 6, om.copy()), FluxPlane(0, nx - pml - 4, om.copy())]
    return Problem(nx, ny, nz, 0.5, periodic=(False, False, False), pml=(pml,) * 6, mat=mat,
                   materials=[Material(1.0), Material(2.25)], sources=src,
                   molecules=pack_molecules(mats), planes=planes,
                   name=f"bragg-{nx}x{ny}x{nz}-{nmol}ml")


def adjoint_design(n: int = 192, design: int = 96, nmol: int = 2000, pml: int = 10, sigma: float = 1.5,
                   gamma: float = 0.02, seed: int = 4, omega: float = 0.25, width: float = 20.0,
                   mol_x: Optional[Tuple[float, float]] = None, multilevel: bool = False,
                   media: bool = False) -> Problem:
    """Inverse-design problem for the adjoint: vacuum cube with CPML on every face, a
    centred design box of `design`^3 cells with eps = 1 + U(0, 1.5), `nmol` two-level
    emitters (omega0 = `omega`, mu12 = 1 along z, coupling `gamma`, ground state) in a
    slab in front of the box, a z-polarised Gaussian-pulse current sheet (carrier
    `omega`, width `width`, peak at 5 widths) on the plane x = pml + 2 and one flux
    plane near the far x face.  The pulse travels along x, so its field and the
    dipoles are both along z.

    `multilevel` makes the emitters RK4 GKSL systems with level count uniform in 2..8
    (harmonic ladders at `omega` +- 5 %, Hermitian z-dipoles with N(0, 0.5) entries,
    log-uniform ladder decay in [1e-5, 1e-3], ground state).  `media` adds behind the
    design box a 4-cell Lorentz layer (eps_inf 1.5, delta_eps 1, omega0 0.3, gamma 0.01)
    and a 2-cell film with a weak Drude pole (wp 0.2, gamma 0.05) plus a Lorentz pole
    (wp 0.1, omega0 0.6, gamma 0.1).  Both draw from a generator of their own, so the
    default problem does not change."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x0 = (n - design) // 2
    deps = 1.0 + rng.uniform(0.0, 1.5, (design, design, design))
    R = int(np.ceil(3 * sigma))
    if mol_x is None:
        mol_x = (max(R + 1.0, x0 - 12.0), max(R + 2.0, x0 - 4.0))
    lo, hi = pml + R + 1.0, n - pml - R - 2.0
    xs = rng.uniform(mol_x[0], mol_x[1], size=nmol)
    ys = rng.uniform(lo, hi, size=nmol)
    zs = rng.uniform(lo, hi, size=nmol)
    if not multilevel:
        mats = [tls((xs[m], ys[m], zs[m]), omega, 1.0, axis=2, sigma=sigma, gamma=gamma, cg=1.0, ce=0.0)
                for m in range(nmol)]
    else:
        r2 = np.random.Generator(np.random.PCG64(seed + 1000))
        nl = r2.integers(2, 9, size=nmol)
        rates = np.exp(r2.uniform(np.log(1e-5), np.log(1e-3), size=nmol))
        mats = []
        for m in range(nmol):
            k = int(nl[m])
            E = np.concatenate([[0.0], np.cumsum(omega * (1 + r2.uniform(-0.05, 0.05, size=k - 1)))])
            mu = np.zeros((3, k, k), np.complex128)
            mu[2] = random_hermitian(r2, k, 0.5)
            rho = np.zeros((k, k), np.complex128)
            rho[0, 0] = 1.0
            mats.append(dict(n=k, pos=(xs[m], ys[m], zs[m]), sigma=sigma, gamma=gamma,
                             H0=np.diag(E).astype(np.complex128), mu=mu, rho=rho,
                             decay=float(rates[m]), kind=KIND_RK4, nsub=1))
    mat, materials = None, [Material(1.0)]
    if media:
        mat = np.zeros((n, n, n), np.uint8)
        xl = x0 + design + 4
        mat[:, :, xl:xl + 4] = 1
        mat[:, :, xl + 4:xl + 6] = 2
        materials = [Material(1.0), Material(1.5, wp=0.3, gamma=0.01, omega0=0.3),
                     Material(1.0, wp=0.2, gamma=0.05, extra=((0.1, 0.1, 0.6),))]
    src = [Source(axis=0, index=pml + 2, comp=2, amp=1.0, omega=omega, width=width, t0=5.0 * width)]
    planes = [FluxPlane(0, n - pml - 4, np.array([omega]))]
    kind = "ml" if multilevel else "tls"
    return Problem(n, n, n, 0.5, pml=(pml,) * 6, design_box=(x0, x0, x0, design, design, design),
                   design_eps=deps, sources=src, molecules=pack_molecules(mats), planes=planes,
                   mat=mat, materials=materials,
                   name=f"adjoint-design-{n}^3-box{design}^3-{nmol}{kind}" + ("-media" if media else ""))


def plasmonic_instance(edge: int, nmol: int, rng, pml: int = 8, omega: float = 0.25, mu12: float = 0.05,
                       sigma: float = 1.5, width: float = 20.0) -> Problem:
    """One realisation of the plasmonic-heating geometry: cube of `edge` cells with CPML
    on every face, a Drude sphere (eps_inf 1, plasma frequency 1, damping 0.05) of
    radius edge/6 at the centre, `nmol` ground-state two-level emitters (omega0
    `omega`, mu12 along z) at positions uniform in volume in the shell r+2 <= |x-c| <=
    r+6, and a z-polarised Gaussian-pulse current sheet on the plane x = pml + 2."""
    n = edge
    r = edge / 6.0
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    c = n / 2.0
    inside = (xx + 0.5 - c) ** 2 + (yy + 0.5 - c) ** 2 + (zz + 0.5 - c) ** 2 < r * r
    mat = np.zeros((n, n, n), np.uint8)
    mat[inside] = 1
    # uniform in the shell volume: radius by inverse CDF of r^2, direction uniform
    r0, r1 = r + 2.0, r + 6.0
    u = rng.uniform(0, 1, nmol)
    rad = (r0 ** 3 + u * (r1 ** 3 - r0 ** 3)) ** (1.0 / 3.0)
    v = rng.normal(size=(nmol, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pos = c + rad[:, None] * v
    mats = [tls(tuple(pos[m]), omega, mu12, axis=2, sigma=sigma, cg=1.0, ce=0.0) for m in range(nmol)]
    src = [Source(axis=0, index=pml + 2, comp=2, amp=1.0, omega=omega, width=width, t0=5.0 * width)]
    return Problem(n, n, n, 0.5, pml=(pml,) * 6, mat=mat,
                   materials=[Material(1.0), Material(1.0, wp=1.0, gamma=0.05)], sources=src,
                   molecules=pack_molecules(mats), name=f"plasmonic-{n}^3-{nmol}tls")


def plasmonic_batch(count: int = 64, seed: int = 5, edges=(64, 96, 128, 160), nmol_range=(200, 5000)) -> List[Problem]:
    """`count` independent realisations: edge drawn uniformly from `edges`, emitter
    count uniform in `nmol_range` (stand-in for the plasmonic-heating ensembles of
    Sec. IV.D as a batch of disorder realisations)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        edge = int(rng.choice(edges))
        nmol = int(rng.integers(nmol_range[0], nmol_range[1] + 1))
        # batched grids fill the GPU together: long z chunks (fewer boundary planes
        # and ring fills per cell) beat the many short ones a lone grid needs
        out.append(plasmonic_instance(edge, nmol, rng).replace(zchunk=32))
    return out


def acceptor_model(rng, omega_e: float, mu_e: float, n: int = 8, pos=(0.0, 0.0, 0.0), sigma: float = 1.5,
                   nsub: int = 1) -> dict:
    """Seeded n-level model acceptor (stand-in for the lowest singlet states of the
    paper's molecular acceptor in Sec. IV.B): ground state 0 and n-1 excited states, one
    of them at omega_e with the strongest transition dipole mu_e from the ground state;
    the others at energies uniform in [0.6, 2.5] omega_e with ground-state dipoles
    U(0.05, 0.4) mu_e and couplings among the excited states N(0, 0.05 mu_e); all dipoles
    along z, real and symmetric; levels sorted by energy; starts in the ground state.
    n = 2 is the single-transition acceptor.  Propagated by RK4 (kind 1)."""
    E = np.concatenate([[omega_e], rng.uniform(0.6, 2.5, size=n - 2) * omega_e]) if n > 2 else np.array([omega_e])
    d0 = np.concatenate([[mu_e], rng.uniform(0.05, 0.4, size=n - 2) * mu_e]) if n > 2 else np.array([mu_e])
    order = np.argsort(E)
    E, d0 = E[order], d0[order]
    mz = np.zeros((n, n))
    mz[0, 1:] = d0
    if n > 2:
        x = rng.normal(0.0, 0.05 * mu_e, size=(n - 1, n - 1))
        mz[1:, 1:] = np.triu(x, 1)
    mz = mz + mz.T
    mu = np.zeros((3, n, n), np.complex128)
    mu[2] = mz
    rho = np.zeros((n, n), np.complex128)
    rho[0, 0] = 1.0
    return dict(n=n, pos=tuple(pos), sigma=sigma, gamma=1.0, H0=np.diag(np.concatenate([[0.0], E])).astype(np.complex128),
                mu=mu, rho=rho, decay=0.0, dephase=0.0, kind=KIND_RK4, nsub=nsub)


def energy_transfer(edge: int = 96, distance: float = 12.0, n_acceptor: int = 8, omega_e: float = 0.25,
                    mu_acceptor: float = 0.02, ratio: float = 100.0, pml: int = 10, seed: int = 11,
                    sigma: float = 1.5) -> Problem:
    """Resonance energy transfer in 3D vacuum (stand-in for the setup of Sec. IV.B): a
    two-level donor (frequency omega_e, dipole ratio * mu_acceptor along z, coherent
    state (1/sqrt 2, 1/sqrt 2)) and an n-level model acceptor (`acceptor_model`) in its
    ground state, `distance` cells apart along x about the centre of an `edge`^3 cube
    with CPML on every face.  In grid units omega_e = 0.25 is a 25-cell wavelength, so
    the paper's 0.04-wavelength separation is below the coupling width; the distance is
    a parameter instead."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = edge / 2.0
    don = tls((c - distance / 2.0, c, c), omega_e, ratio * mu_acceptor, axis=2, sigma=sigma,
              cg=np.sqrt(0.5), ce=np.sqrt(0.5))
    acc = acceptor_model(rng, omega_e, mu_acceptor, n_acceptor, pos=(c + distance / 2.0, c, c), sigma=sigma)
    return Problem(edge, edge, edge, 0.5, pml=(pml,) * 6, molecules=pack_molecules([don, acc]),
                   name=f"energy-transfer-{edge}^3-d{distance:g}-n{n_acceptor}")


def energy_transfer_batch(count: int = 64, edge: int = 96, seed: int = 12, distances=(8.0, 24.0),
                          models=(2, 4, 8)) -> List[Problem]:
    """`count` independent donor-acceptor realisations: distance uniform in `distances`,
    acceptor level count drawn from `models` (the single-transition acceptor against
    multilevel models, as Sec. IV.B compares them), each with its own seeded model."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for q in range(count):
        d = float(rng.uniform(*distances))
        n = int(rng.choice(models))
        out.append(energy_transfer(edge=edge, distance=d, n_acceptor=n, seed=seed * 1000 + q).replace(zchunk=32))
    return out


def small_coupled(seed: int = 0, shape=(24, 20, 28), nmol: int = 6, pml: int = 4,
                  multilevel: bool = True, eps_map: bool = True, drude: bool = False,
                  source: bool = True, planes: bool = True, periodic=(False, False, False),
                  lorentz: bool = False) -> Problem:
    """Small ragged problem for parity tests: every feature at once on a grid the
    oracle finishes in well under a second per hundred steps.  `drude` puts a Drude
    sphere at the centre; `lorentz` (with `drude`) turns its upper half (z above the
    centre) into a three-pole medium (two Lorentz oscillators and a Drude term), so that
    one pole box holds one- and three-pole cells."""
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    nx, ny, nz = shape
    pmls = tuple(0 if periodic[a // 2] else pml for a in range(6))
    mat = None
    materials = [Material(1.0)]
    design_box = None
    design_eps = None
    if eps_map:
        mat = np.zeros((nz, ny, nx), np.uint8)
        materials.append(Material(2.25))
        mat[nz // 2 + 3:nz // 2 + 6] = 1
        sx, sy, sz = max(2, nx // 4), max(2, ny // 4), max(2, nz // 5)
        design_box = (nx // 2 - sx // 2, ny // 2 - sy // 2, 2 + pml, sx, sy, sz)
        design_eps = 1.0 + rng.uniform(0, 1.5, size=(sz, sy, sx))
    if drude:
        if mat is None:
            mat = np.zeros((nz, ny, nx), np.uint8)
        materials.append(Material(1.0, wp=1.0, gamma=0.05))
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        r = min(nx, ny, nz) / 6
        inside = (xx + 0.5 - nx / 2) ** 2 + (yy + 0.5 - ny / 2) ** 2 + (zz + 0.5 - nz / 2) ** 2 < r * r
        mat[inside] = len(materials) - 1
        if lorentz:
            materials.append(Material(1.5, wp=0.6, gamma=0.02, omega0=0.3,
                                      extra=((0.4, 0.05, 0.55), (0.3, 0.1, 0.0))))
            mat[inside & (zz >= nz // 2)] = len(materials) - 1
    mats = []
    for m in range(nmol):
        sigma = float(rng.choice([1.0, 1.5]))
        R = int(np.ceil(3 * sigma))
        p = []
        for a, n in enumerate(shape):
            if periodic[a]:
                p.append(rng.uniform(0, n))
            else:
                p.append(rng.uniform(R + 1, n - R - 2))
        if multilevel and m % 2 == 1:
            n = int(rng.integers(3, 9))
            steps = 0.2 * (1 + rng.uniform(-0.05, 0.05, size=n - 1))
            E = np.concatenate([[0.0], np.cumsum(steps)])
            mu = np.stack([random_hermitian(rng, n, 0.3) for _ in range(3)])
            c = rng.normal(size=n) + 1j * rng.normal(size=n)
            c /= np.linalg.norm(c)
            mats.append(dict(n=n, pos=tuple(p), sigma=sigma, gamma=float(rng.uniform(0.5, 1.5)),
                             H0=np.diag(E).astype(np.complex128), mu=mu,
                             rho=np.outer(c, c.conj()), decay=float(rng.uniform(0, 1e-2)),
                             dephase=float(rng.uniform(0, 1e-2)), kind=KIND_RK4,
                             nsub=int(rng.integers(1, 3))))
        else:
            ce = np.sqrt(rng.uniform(0.05, 0.95))
            cg = np.sqrt(1 - ce ** 2) * np.exp(1j * rng.uniform(0, 2 * np.pi))
            mats.append(tls(tuple(p), 0.25, float(rng.uniform(0.2, 1.0)), axis=int(rng.integers(0, 3)),
                            sigma=sigma, gamma=float(rng.uniform(0.5, 1.5)), cg=cg, ce=ce))
    srcs = []
    if source:
        srcs.append(Source(axis=2, index=pmls[4] + 2 if not periodic[2] else 1, comp=0, amp=0.5,
                           omega=0.3, width=6.0, t0=18.0))
    pl = []
    if planes:
        om = np.linspace(0.2, 0.35, 3)
        pl.append(FluxPlane(2, nz - pmls[5] - 2, om.copy()))
        pl.append(FluxPlane(0, pmls[0] + 2, om.copy()))
        pl.append(FluxPlane(1, ny // 2, om.copy()))
    return Problem(nx, ny, nz, 0.5, periodic=tuple(periodic), pml=pmls, mat=mat,
                   materials=materials, design_box=design_box, design_eps=design_eps,
                   sources=srcs, molecules=pack_molecules(mats) if mats else empty_molecules(),
                   planes=pl, name=f"small-{nx}x{ny}x{nz}-s{seed}")


def random_fields(prob: Problem, seed: int, scale: float = 1.0):
    """Seeded random initial E and H (6 arrays of shape (nz, ny, nx), float64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [scale * rng.standard_normal((prob.nz, prob.ny, prob.nx)) for _ in range(6)]


def cavity_ensemble(M: int = 1_000_000, omega0: float = 0.25, mu12: float = 0.05, seed: int = 6) -> Molecules:
    """Single-mode cavity workload (stand-in for the normal-mode examples of Sec. II):
    `M` two-level emitters (H0 = diag(0, omega0), exact propagator), transition dipole
    mu12 sigma_x in the cavity plane at a seeded uniform angle, gamma = 1, ground state
    with a seeded 1e-3 coherence.  Built with array operations (pools of 4 elements per
    emitter at offset 4 m)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = rng.uniform(0.0, 2 * np.pi, M)
    ph = rng.uniform(0.0, 2 * np.pi, M)
    cg, ce = np.sqrt(1.0 - 1e-6), 1e-3 * np.exp(1j * ph)
    H0 = np.zeros((M, 4), np.complex128)
    H0[:, 3] = omega0
    mu = np.zeros((3, M, 4), np.complex128)
    mu[0, :, 1] = mu[0, :, 2] = mu12 * np.cos(th)
    mu[1, :, 1] = mu[1, :, 2] = mu12 * np.sin(th)
    rho = np.stack([np.full(M, cg * cg), cg * np.conj(ce), ce * cg, np.abs(ce) ** 2], axis=1).astype(np.complex128)
    return Molecules(np.full(M, 2, np.int32), 4 * np.arange(M, dtype=np.int64), np.zeros((M, 3)),
                     np.ones(M), np.ones(M), np.zeros(M), np.zeros(M), np.zeros(M, np.int32),
                     np.ones(M, np.int32), H0.ravel(), mu.reshape(3, -1), rho.ravel())

