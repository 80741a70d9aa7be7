"""FP64 CPU oracle for the coupled Yee / molecular-ensemble step (test infrastructure).

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may
import this package.  It wraps `maxlink_oracle.c` (plain C, FP64) through ctypes and
converts a `Problem` description into the oracle's full-grid arrays by itself; it
shares no code with the CUDA library.

Functions without an independent pin are marked "parity unpinned" in their
docstring (none at present: every piece is pinned by a test under `tests/`,
see `tests/test_oracle_*.py`; the discrete adjoint by a dot-product identity and
central differences in `tests/test_oracle_adjoint.py`; the single-mode cavity of
`oracle/cavity.py` in `tests/test_oracle_cavity.py`; the laser-driven molecules of
`oracle/laser.py` in `tests/test_oracle_laser.py`).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "maxlink_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmaxlink_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP on independent cell loops only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    L = C.CDLL(_LIB)
    P = C.c_void_p
    dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    L.orc_create.restype = P
    L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, ip, ip, C.c_double, C.c_double,
                             C.c_double, C.c_double, P, C.c_int, P, P, P]
    L.orc_destroy.argtypes = [P]
    L.orc_add_molecule.restype = C.c_int
    L.orc_add_molecule.argtypes = [P, C.c_int, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_int, C.c_int, dp, dp, dp]
    L.orc_step.restype = C.c_int
    L.orc_step.argtypes = [P, C.c_long]
    L.orc_add_source.restype = C.c_int
    L.orc_add_source.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                 C.c_double]
    L.orc_add_plane.restype = C.c_int
    L.orc_add_plane.argtypes = [P, C.c_int, C.c_int, C.c_int, dp]
    L.orc_flux.restype = C.c_int
    L.orc_flux.argtypes = [P, C.c_int, dp]
    L.orc_plane_data.restype = C.c_int
    L.orc_plane_data.argtypes = [P, C.c_int, dp]
    L.orc_get_fields.argtypes = [P, dp]
    L.orc_set_fields.argtypes = [P, dp]
    L.orc_get_drude.argtypes = [P, dp]
    L.orc_get_psi.argtypes = [P, dp]
    L.orc_get_current.argtypes = [P, dp]
    L.orc_nmol.restype = C.c_int
    L.orc_nmol.argtypes = [P]
    L.orc_step_count.restype = C.c_long
    L.orc_step_count.argtypes = [P]
    L.orc_absorbed.restype = C.c_double
    L.orc_absorbed.argtypes = [P]
    L.orc_get_mol.restype = C.c_int
    L.orc_get_mol.argtypes = [P, C.c_int, dp, dp, dp]
    L.orc_get_rho.restype = C.c_int
    L.orc_get_rho.argtypes = [P, C.c_int, dp]
    L.orc_set_rho.restype = C.c_int
    L.orc_set_rho.argtypes = [P, C.c_int, dp]
    L.orc_gather.restype = C.c_int
    L.orc_gather.argtypes = [P, C.c_int, dp]
    L.orc_molecule_step.restype = C.c_int
    L.orc_molecule_step.argtypes = [P, C.c_int, dp, C.c_double, dp]
    L.orc_lindblad_rhs.restype = C.c_int
    L.orc_lindblad_rhs.argtypes = [P, C.c_int, dp, dp, dp]
    L.orc_pml_tables.argtypes = [P, C.c_int, dp]
    L.orc_set_psi.argtypes = [P, dp]
    L.orc_set_drude.argtypes = [P, dp]
    L.orc_adj_reset.argtypes = [P]
    L.orc_adj_get.argtypes = [P, dp]
    L.orc_adj_set.argtypes = [P, dp]
    L.orc_npole.restype = C.c_int
    L.orc_npole.argtypes = [P]
    L.orc_get_poles.argtypes = [P, dp]
    L.orc_set_poles.argtypes = [P, dp]
    L.orc_adj_field.argtypes = [P]
    L.orc_mol_vjp.restype = C.c_int
    L.orc_mol_vjp.argtypes = [P, C.c_int, dp, dp, dp, dp, dp, dp]
    L.orc_adjoint_run.restype = C.c_int
    L.orc_adjoint_run.argtypes = [P, C.c_long, C.c_int, C.c_int, dp, dp, dp]
    L.orc_threads.restype = C.c_int
    L.orc_threads.argtypes = []
    _lib = L
    return L


def _ri(z: np.ndarray) -> np.ndarray:
    z = np.ascontiguousarray(z, dtype=np.complex128)
    return np.ascontiguousarray(z.view(np.float64).ravel())


def threads() -> int:
    return int(_load().orc_threads())


class OracleSim:
    """FP64 oracle instance built from a `workloads.Problem`."""

    def __init__(self, prob, molecules: bool = True):
        L = _load()
        self.L = L
        self.prob = prob
        nx, ny, nz = prob.nx, prob.ny, prob.nz
        self.shape = (nz, ny, nx)
        N = nx * ny * nz
        # material description -> full-grid eps and, per pole slot, strength, damping and
        # resonance (own conversion); a material's poles take slots 0, 1, ... in order
        mats = prob.materials
        npole = max([1] + [len(mt.poles()) for mt in mats])
        eps = np.ones(self.shape)
        wp = np.zeros((npole,) + self.shape)
        dg = np.zeros((npole,) + self.shape)
        w0 = np.zeros((npole,) + self.shape)
        idx = np.asarray(prob.mat) if prob.mat is not None else np.zeros(self.shape, np.uint8)
        for q, mt in enumerate(mats):
            sel = idx == q
            eps[sel] = mt.eps_inf
            for p, (a, g, r) in enumerate(mt.poles()):
                wp[p][sel] = a
                dg[p][sel] = g
                w0[p][sel] = r
        if prob.design_box is not None:
            x0, y0, z0, sx, sy, sz = prob.design_box
            eps[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx] = prob.design_eps
        self._eps = np.ascontiguousarray(eps.ravel())
        self._wp = np.ascontiguousarray(wp.ravel())
        self._dg = np.ascontiguousarray(dg.ravel())
        self._w0 = np.ascontiguousarray(w0.ravel())
        per = np.array([1 if p else 0 for p in prob.periodic], np.int32)
        pml = np.array(prob.pml, np.int32)
        self.h = L.orc_create(nx, ny, nz, prob.dt, per, pml, prob.pml_m, prob.pml_sigma_max,
                              prob.pml_kappa_max, prob.pml_alpha_max,
                              self._eps.ctypes.data, npole, self._wp.ctypes.data, self._dg.ctypes.data,
                              self._w0.ctypes.data)
        if not self.h:
            raise ValueError(f"oracle: {npole} poles per material is more than it holds")
        for s in prob.sources:
            L.orc_add_source(self.h, s.axis, s.index, s.comp, s.amp, s.omega, s.width, s.t0)
        for p in prob.planes:
            L.orc_add_plane(self.h, p.axis, p.index, len(p.omegas),
                            np.ascontiguousarray(p.omegas, np.float64))
        if molecules:
            mol = prob.molecules
            for m in range(mol.count):
                n = int(mol.nlev[m])
                mu = np.stack([mol.matrix(mol.mu[a], m) for a in range(3)])
                r = L.orc_add_molecule(self.h, n, np.ascontiguousarray(mol.pos[m], np.float64),
                                       float(mol.sigma[m]), float(mol.gamma[m]),
                                       float(mol.decay[m]), float(mol.dephase[m]),
                                       int(mol.kind[m]), int(mol.nsub[m]),
                                       _ri(mol.matrix(mol.H0, m)), _ri(mu),
                                       _ri(mol.matrix(mol.rho0, m)))
                if r < 0:
                    raise ValueError("bad molecule")

    def __del__(self):
        if getattr(self, "h", None):
            self.L.orc_destroy(self.h)
            self.h = None

    # -- stepping and state ------------------------------------------------------
    def step(self, n: int = 1):
        if self.L.orc_step(self.h, int(n)) != 0:
            raise ValueError("molecule window outside a non-periodic grid")

    @property
    def nstep(self) -> int:
        return int(self.L.orc_step_count(self.h))

    def fields(self) -> List[np.ndarray]:
        N = int(np.prod(self.shape))
        out = np.zeros(6 * N)
        self.L.orc_get_fields(self.h, out)
        return [out[q * N:(q + 1) * N].reshape(self.shape) for q in range(6)]

    def set_fields(self, f: List[np.ndarray]):
        buf = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).ravel() for x in f]))
        self.L.orc_set_fields(self.h, buf)

    def drude_current(self):
        N = int(np.prod(self.shape))
        out = np.zeros(3 * N)
        self.L.orc_get_drude(self.h, out)
        return [out[q * N:(q + 1) * N].reshape(self.shape) for q in range(3)]

    def psi(self):
        N = int(np.prod(self.shape))
        out = np.zeros(12 * N)
        self.L.orc_get_psi(self.h, out)
        return [out[q * N:(q + 1) * N].reshape(self.shape) for q in range(12)]

    def current(self):
        N = int(np.prod(self.shape))
        out = np.zeros(3 * N)
        self.L.orc_get_current(self.h, out)
        return [out[q * N:(q + 1) * N].reshape(self.shape) for q in range(3)]

    @property
    def nmol(self) -> int:
        return int(self.L.orc_nmol(self.h))

    def mol_state(self, m: int):
        Et, md, es = np.zeros(3), np.zeros(3), np.zeros(1)
        self.L.orc_get_mol(self.h, m, Et, md, es)
        return Et, md, float(es[0])

    def rho(self, m: int) -> np.ndarray:
        buf = np.zeros(2 * 64)
        n = self.L.orc_get_rho(self.h, m, buf)
        return buf[:2 * n * n].view(np.complex128).reshape(n, n).copy()

    def set_rho(self, m: int, rho: np.ndarray):
        self.L.orc_set_rho(self.h, m, _ri(rho))

    def populations(self) -> List[np.ndarray]:
        return [np.real(np.diag(self.rho(m))) for m in range(self.nmol)]

    def gather(self, m: int) -> np.ndarray:
        out = np.zeros(3)
        if self.L.orc_gather(self.h, m, out) != 0:
            raise ValueError("window outside grid")
        return out

    def molecule_step(self, m: int, Et, dt: Optional[float] = None) -> np.ndarray:
        md = np.zeros(3)
        self.L.orc_molecule_step(self.h, m, np.ascontiguousarray(Et, np.float64),
                                 self.prob.dt if dt is None else float(dt), md)
        return md

    def lindblad_rhs(self, m: int, Et, rho: np.ndarray) -> np.ndarray:
        n = rho.shape[0]
        out = np.zeros(2 * n * n)
        self.L.orc_lindblad_rhs(self.h, m, np.ascontiguousarray(Et, np.float64), _ri(rho), out)
        return out.view(np.complex128).reshape(n, n)

    def flux(self, p: int) -> np.ndarray:
        out = np.zeros(len(self.prob.planes[p].omegas))
        self.L.orc_flux(self.h, p, out)
        return out

    def plane_data(self, p: int):
        pl = self.prob.planes[p]
        a = pl.axis
        dims = [self.prob.nx, self.prob.ny, self.prob.nz]
        nb, nc = dims[(a + 1) % 3], dims[(a + 2) % 3]
        cnt = len(pl.omegas) * nb * nc
        out = np.zeros(8 * cnt)
        self.L.orc_plane_data(self.h, p, out)
        z = out.view(np.complex128)
        return [z[q * cnt:(q + 1) * cnt].reshape(len(pl.omegas), nc, nb) for q in range(4)]

    def absorbed(self) -> float:
        return float(self.L.orc_absorbed(self.h))

    def pml_tables(self, axis: int) -> np.ndarray:
        n = [self.prob.nx, self.prob.ny, self.prob.nz][axis]
        out = np.zeros(6 * n)
        self.L.orc_pml_tables(self.h, axis, out)
        return out.reshape(6, n)

    # -- discrete adjoint (reverse mode of `step`) ---------------------------------
    def set_psi(self, psi: List[np.ndarray]):
        self.L.orc_set_psi(self.h, np.ascontiguousarray(np.concatenate([np.ravel(x) for x in psi]), np.float64))

    def set_drude_current(self, jd: List[np.ndarray]):
        self.L.orc_set_drude(self.h, np.ascontiguousarray(np.concatenate([np.ravel(x) for x in jd]), np.float64))

    def adj_reset(self):
        self.L.orc_adj_reset(self.h)

    @property
    def npole(self) -> int:
        return int(self.L.orc_npole(self.h))

    def poles(self) -> List[np.ndarray]:
        """Every pole slot's state: per slot J[3] (at n-1/2) then P[3] (at n)."""
        N = int(np.prod(self.shape))
        out = np.zeros(6 * self.npole * N)
        self.L.orc_get_poles(self.h, out)
        return [out[q * N:(q + 1) * N].reshape(self.shape) for q in range(6 * self.npole)]

    def set_poles(self, st: List[np.ndarray]):
        self.L.orc_set_poles(self.h, np.ascontiguousarray(np.concatenate([np.ravel(x) for x in st]), np.float64))

    def adj_state(self) -> np.ndarray:
        """Adjoint field state as (18 + 6 npole, nz, ny, nx): Eb[3], Hb[3], psi_b[12], then
        per pole slot J_b[3], P_b[3]."""
        N = int(np.prod(self.shape))
        n = 18 + 6 * self.npole
        out = np.zeros(n * N)
        self.L.orc_adj_get(self.h, out)
        return out.reshape((n,) + self.shape)

    def set_adj_state(self, st: np.ndarray):
        self.L.orc_adj_set(self.h, np.ascontiguousarray(st, np.float64).ravel())

    def adj_field_step(self):
        """Transpose of the field part of one step (CPML H and E updates, Drude)."""
        self.L.orc_adj_field(self.h)

    def mol_vjp(self, m: int, Et, rho: np.ndarray, X: np.ndarray, mdb):
        """Adjoints of (rho, Et) of one molecule step (exact two-level or RK4 GKSL) from
        those of (rho', mudot)."""
        n = rho.shape[0]
        rb = np.zeros(2 * n * n)
        Etb = np.zeros(3)
        if self.L.orc_mol_vjp(self.h, m, np.ascontiguousarray(Et, np.float64), _ri(rho), _ri(X),
                              np.ascontiguousarray(mdb, np.float64), rb, Etb) != 0:
            raise ValueError("bad molecule index")
        return rb.view(np.complex128).reshape(n, n), Etb

    def adjoint_run(self, nsteps: int, plane: int, freq: int):
        """Run nsteps from the present state; return the flux of `plane` at frequency
        index `freq` over those steps and its gradients with respect to the
        permittivity of every cell (nz, ny, nx) and the coupling of every molecule."""
        N = int(np.prod(self.shape))
        ge = np.zeros(N)
        gg = np.zeros(max(self.nmol, 1))
        obj = np.zeros(1)
        rc = self.L.orc_adjoint_run(self.h, int(nsteps), int(plane), int(freq), ge, gg, obj)
        if rc != 0:
            raise ValueError(f"adjoint run failed ({rc})")
        return float(obj[0]), ge.reshape(self.shape), gg[:self.nmol]
