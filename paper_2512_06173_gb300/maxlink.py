"""ctypes binding of libmaxlink (include/maxlink.h), argument marshalling only.

Every entry point of the C ABI is exposed under its own name (`ml_grid_create`,
`ml_add_molecules`, `ml_step`, `ml_get_fields`, `ml_flux`, ...).  `Grid` wraps a
handle built from a `workloads.Problem`.  All computation happens in the CUDA
library; if it cannot be loaded this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional

import numpy as np

from . import build as _build

ML_OK, ML_ERR_INVALID_ARG, ML_ERR_CUDA, ML_ERR_OOM, ML_ERR_STATE, ML_ERR_TIMEOUT, ML_ERR_NUMERIC = range(7)
ML_F32, ML_F64 = 0, 1
ML_MOL_RHO, ML_MOL_EFIELD, ML_MOL_MUDOT, ML_MOL_ENERGY, ML_MOL_POP = range(5)
ML_EX, ML_EY, ML_EZ, ML_HX, ML_HY, ML_HZ, ML_ALL = 1, 2, 4, 8, 16, 32, 63
ML_MAX_LEVELS = 8
ML_HOST_ASYNC = 2  # ml_get_molecules: page-locked host destination, no synchronisation
ML_STATIC_GATHER_MAX_MOLECULES = 16384

EXPORTED = ["ml_last_error", "ml_version", "ml_grid_create", "ml_grid_destroy", "ml_add_molecules",
            "ml_add_flux_plane", "ml_step", "ml_get_fields", "ml_set_fields", "ml_get_molecules", "ml_flux",
            "ml_flux_data", "ml_absorbed", "ml_sync_status", "ml_step_count", "ml_molecule_count",
            "ml_checkpoint", "ml_restore", "ml_set_timing", "ml_timing", "ml_launch_count"]


ML_MAX_POLES = 4


class ml_pole(C.Structure):
    _fields_ = [("wp", C.c_double), ("gamma", C.c_double), ("omega0", C.c_double)]


class ml_material(C.Structure):
    _fields_ = [("eps_inf", C.c_double), ("wp", C.c_double), ("gamma", C.c_double), ("omega0", C.c_double),
                ("n_extra", C.c_int), ("extra", ml_pole * (ML_MAX_POLES - 1))]


def _material(x) -> ml_material:
    """workloads.Material -> ml_material (first pole, then the extra ones)."""
    m = ml_material(x.eps_inf, x.wp, x.gamma, x.omega0)
    if len(x.extra) > ML_MAX_POLES - 1:
        raise ValueError(f"at most {ML_MAX_POLES} poles per material")
    m.n_extra = len(x.extra)
    for q, (wp, g, w0) in enumerate(x.extra):
        m.extra[q] = ml_pole(wp, g, w0)
    return m


class ml_source(C.Structure):
    _fields_ = [("axis", C.c_int), ("index", C.c_int), ("comp", C.c_int), ("amp", C.c_double),
                ("omega", C.c_double), ("width", C.c_double), ("t0", C.c_double)]


class ml_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("courant", C.c_double),
                ("precision", C.c_int), ("periodic", C.c_int * 3), ("pml", C.c_int * 6),
                ("pml_m", C.c_double), ("pml_sigma_max", C.c_double), ("pml_kappa_max", C.c_double),
                ("pml_alpha_max", C.c_double), ("mat", C.c_void_p), ("n_materials", C.c_int),
                ("materials", C.POINTER(ml_material)), ("design_box", C.c_int * 6),
                ("design_eps", C.c_void_p), ("n_sources", C.c_int), ("sources", C.POINTER(ml_source)),
                ("zchunk", C.c_int)]


class ml_molecule_desc(C.Structure):
    _fields_ = [("count", C.c_int), ("nlev", C.c_void_p), ("off", C.c_void_p), ("pos", C.c_void_p),
                ("sigma", C.c_void_p), ("gamma", C.c_void_p), ("decay", C.c_void_p), ("dephase", C.c_void_p),
                ("kind", C.c_void_p), ("nsub", C.c_void_p), ("H0", C.c_void_p), ("mu", C.c_void_p),
                ("rho", C.c_void_p), ("pool", C.c_int64)]


class ml_cavity_desc(C.Structure):
    _fields_ = [("omega_c", C.c_double), ("coupling", C.c_double), ("dt", C.c_double),
                ("q0", C.c_double * 2), ("p0", C.c_double * 2), ("precision", C.c_int)]


class ml_drive_desc(C.Structure):
    _fields_ = [("amplitude", C.c_double), ("omega", C.c_double), ("phase", C.c_double), ("center", C.c_double),
                ("half_width", C.c_double), ("polarization", C.c_double * 3), ("dt", C.c_double),
                ("precision", C.c_int)]


_lib = None

# ml_alloc_fn / ml_free_fn of the header
_ALLOC_T = C.CFUNCTYPE(C.c_int, C.POINTER(C.c_void_p), C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_T = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class TorchAllocator:
    """The boundary's allocator callback backed by PyTorch's caching allocator: every
    device buffer the library allocates comes from `torch.cuda.caching_allocator_alloc`
    and goes back through `torch.cuda.caching_allocator_delete`.  Counts the calls and
    the bytes the library holds."""

    def __init__(self):
        self.allocs = 0
        self.frees = 0
        self.live_bytes = 0
        self.c_alloc = _ALLOC_T(self._alloc)
        self.c_free = _FREE_T(self._free)

    def _alloc(self, pp, nbytes, stream, ctx):
        try:
            import torch
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except Exception:
            return 1
        pp[0] = ptr
        self.allocs += 1
        self.live_bytes += int(nbytes)
        return 0

    def _free(self, ptr, nbytes, stream, ctx):
        try:
            import torch
            torch.cuda.caching_allocator_delete(int(ptr))
        finally:
            self.frees += 1
            self.live_bytes -= int(nbytes)


_allocator: Optional[TorchAllocator] = None


class MaxlinkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"maxlink status {status}: {msg}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmaxlink.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        try:
            path = _build.build()
        except Exception as e:  # no toolkit: only an existing library can be used
            if not os.path.exists(path):
                raise RuntimeError(f"libmaxlink is not built and cannot be built: {e}") from e
    if not os.path.exists(path):
        raise RuntimeError(f"libmaxlink not found at {path}")
    L = C.CDLL(path)
    P, I, I64, D = C.c_void_p, C.c_int, C.c_int64, C.c_double
    sig = {
        "ml_last_error": (C.c_char_p, []),
        "ml_version": (C.c_char_p, []),
        "ml_grid_create": (I, [C.POINTER(ml_grid_desc), P, C.POINTER(P)]),
        "ml_grid_destroy": (I, [P]),
        "ml_add_molecules": (I, [P, C.POINTER(ml_molecule_desc), P, C.POINTER(I)]),
        "ml_add_flux_plane": (I, [P, I, I, I, P, C.POINTER(I)]),
        "ml_step": (I, [P, I64, P]),
        "ml_get_fields": (I, [P, C.c_uint, P, I, P]),
        "ml_set_fields": (I, [P, C.c_uint, P, I, P]),
        "ml_get_molecules": (I, [P, I, P, I, P]),
        "ml_set_population_sink": (I, [P, P, I64]),
        "ml_flux": (I, [P, I, P, P]),
        "ml_flux_data": (I, [P, I, P, P]),
        "ml_absorbed": (I, [P, P, P]),
        "ml_sync_status": (I, [P, P]),
        "ml_set_wait_limit": (I, [P, I64]),
        "ml_set_allocator": (I, [_ALLOC_T, _FREE_T, P]),
        "ml_step_count": (I64, [P]),
        "ml_molecule_count": (I, [P]),
        "ml_checkpoint": (I, [P, P, C.POINTER(C.c_size_t), P]),
        "ml_restore": (I, [P, P, C.c_size_t, P]),
        "ml_set_timing": (I, [P, I]),
        "ml_timing": (I, [P, P, P]),
        "ml_launch_count": (I64, [P]),
        "ml_gather_static": (I, [P, I, I, I, P, I, P, P, P, P, P]),
        "ml_adjoint_run": (I, [P, I64, I, I, I, P, P, P, I, P]),
        "ml_set_design_eps": (I, [P, P, I, P]),
        "ml_set_couplings": (I, [P, P, I, P]),
        "ml_cavity_create": (I, [C.POINTER(ml_cavity_desc), C.POINTER(ml_molecule_desc), C.POINTER(P)]),
        "ml_cavity_destroy": (I, [P]),
        "ml_cavity_step": (I, [P, I64, P]),
        "ml_cavity_mode": (I, [P, P, P]),
        "ml_cavity_get_molecules": (I, [P, I, P, P]),
        "ml_cavity_step_count": (I64, [P]),
        "ml_drive_create": (I, [C.POINTER(ml_drive_desc), C.POINTER(ml_molecule_desc), C.POINTER(P)]),
        "ml_drive_destroy": (I, [P]),
        "ml_drive_step": (I, [P, I64, P]),
        "ml_drive_get_molecules": (I, [P, I, P, P]),
        "ml_drive_step_count": (I64, [P]),
        "ml_batch_create": (I, [P, I, C.POINTER(P)]),
        "ml_batch_step": (I, [P, I64, P]),
        "ml_batch_set_tuning": (I, [P, I, I]),
        "ml_batch_autotune": (I, [P, I, P, C.POINTER(I), C.POINTER(D)]),
        "ml_batch_launch_count": (I64, [P]),
        "ml_batch_set_timing": (I, [P, I]),
        "ml_batch_timing": (I, [P, P, P]),
        "ml_batch_destroy": (I, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    # device memory of the library from PyTorch's caching allocator when a GPU is present
    try:
        import torch
        if torch.cuda.is_available() and os.environ.get("ML_ALLOCATOR", "torch") == "torch":
            use_torch_allocator()
    except ImportError:
        pass
    return L


def ml_set_allocator(alloc=None, free=None, ctx=None):
    """Install ctypes callbacks of types `_ALLOC_T` / `_FREE_T` as the library's device
    allocator (None, None: the library default).  The caller keeps the callbacks alive."""
    _check(load().ml_set_allocator(alloc if alloc is not None else _ALLOC_T(),
                                   free if free is not None else _FREE_T(), ctx))


def use_torch_allocator() -> TorchAllocator:
    """Install (once) the PyTorch-backed allocator and return it."""
    global _allocator
    L = load()
    if _allocator is None:
        a = TorchAllocator()
        _check(L.ml_set_allocator(a.c_alloc, a.c_free, None))
        _allocator = a
    return _allocator


def use_default_allocator():
    """Back to the library's default allocator (cudaMallocAsync / cudaFreeAsync).  Buffers
    allocated before keep going back to the allocator they came from."""
    global _allocator
    _check(load().ml_set_allocator(_ALLOC_T(), _FREE_T(), None))
    if _allocator is not None:
        _keep_alive.append(_allocator)
    _allocator = None


_keep_alive: List[TorchAllocator] = []  # allocators whose buffers may still be alive


def allocator() -> Optional[TorchAllocator]:
    """The PyTorch-backed allocator in use, or None (library default)."""
    return _allocator


def _check(status: int):
    if status != ML_OK:
        msg = load().ml_last_error().decode()
        raise MaxlinkError(status, msg)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---------------------------------------------------------------- C-ABI names

def ml_version() -> str:
    return load().ml_version().decode()


def ml_last_error() -> str:
    return load().ml_last_error().decode()


def ml_grid_create(desc: ml_grid_desc, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(load().ml_grid_create(C.byref(desc), C.c_void_p(stream), C.byref(h)))
    return h.value


def ml_grid_destroy(h: int):
    _check(load().ml_grid_destroy(C.c_void_p(h)))


def ml_add_molecules(h: int, desc: ml_molecule_desc, stream: int = 0) -> int:
    first = C.c_int()
    _check(load().ml_add_molecules(C.c_void_p(h), C.byref(desc), C.c_void_p(stream), C.byref(first)))
    return first.value


def ml_add_flux_plane(h: int, axis: int, index: int, omegas) -> int:
    om = np.ascontiguousarray(omegas, np.float64)
    pid = C.c_int()
    _check(load().ml_add_flux_plane(C.c_void_p(h), axis, index, len(om), C.c_void_p(_ptr(om)), C.byref(pid)))
    return pid.value


def ml_step(h: int, nsteps: int, stream: int = 0):
    _check(load().ml_step(C.c_void_p(h), int(nsteps), C.c_void_p(stream)))


def ml_get_fields(h: int, mask: int, dst_ptr: int, on_device: bool, stream: int = 0):
    _check(load().ml_get_fields(C.c_void_p(h), mask, C.c_void_p(dst_ptr), int(on_device), C.c_void_p(stream)))


def ml_set_fields(h: int, mask: int, src_ptr: int, on_device: bool, stream: int = 0):
    _check(load().ml_set_fields(C.c_void_p(h), mask, C.c_void_p(src_ptr), int(on_device), C.c_void_p(stream)))


def ml_get_molecules(h: int, what: int, dst_ptr: int, on_device: int, stream: int = 0):
    _check(load().ml_get_molecules(C.c_void_p(h), what, C.c_void_p(dst_ptr), int(on_device), C.c_void_p(stream)))


def ml_set_population_sink(h: int, host_ptr: int, ring_steps: int):
    """host_ptr: page-locked host memory (0 removes the sink)."""
    _check(load().ml_set_population_sink(C.c_void_p(h), C.c_void_p(host_ptr), int(ring_steps)))


def ml_flux(h: int, plane: int, nfreq: int, stream: int = 0) -> np.ndarray:
    out = np.zeros(nfreq)
    _check(load().ml_flux(C.c_void_p(h), plane, C.c_void_p(_ptr(out)), C.c_void_p(stream)))
    return out


def ml_flux_data(h: int, plane: int, count: int, stream: int = 0) -> np.ndarray:
    out = np.zeros(2 * count)
    _check(load().ml_flux_data(C.c_void_p(h), plane, C.c_void_p(_ptr(out)), C.c_void_p(stream)))
    return out.view(np.complex128)


def ml_absorbed(h: int, stream: int = 0) -> float:
    out = np.zeros(1)
    _check(load().ml_absorbed(C.c_void_p(h), C.c_void_p(_ptr(out)), C.c_void_p(stream)))
    return float(out[0])


def ml_sync_status(h: int, stream: int = 0):
    _check(load().ml_sync_status(C.c_void_p(h), C.c_void_p(stream)))


def ml_sync_status_code(h: int, stream: int = 0) -> int:
    """The latched device status as an integer (ML_OK, ML_ERR_TIMEOUT, ML_ERR_NUMERIC ...),
    without raising."""
    return int(load().ml_sync_status(C.c_void_p(h), C.c_void_p(stream)))


def ml_set_wait_limit(h: int, probes: int):
    _check(load().ml_set_wait_limit(C.c_void_p(h), int(probes)))


def ml_step_count(h: int) -> int:
    return int(load().ml_step_count(C.c_void_p(h)))


def ml_molecule_count(h: int) -> int:
    return int(load().ml_molecule_count(C.c_void_p(h)))


def ml_checkpoint(h: int, stream: int = 0) -> bytes:
    n = C.c_size_t(0)
    _check(load().ml_checkpoint(C.c_void_p(h), None, C.byref(n), C.c_void_p(stream)))
    buf = C.create_string_buffer(n.value)
    _check(load().ml_checkpoint(C.c_void_p(h), buf, C.byref(n), C.c_void_p(stream)))
    return buf.raw


def ml_restore(h: int, blob: bytes, stream: int = 0):
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().ml_restore(C.c_void_p(h), buf, len(blob), C.c_void_p(stream)))


def ml_set_timing(h: int, enable: bool):
    _check(load().ml_set_timing(C.c_void_p(h), int(enable)))


def ml_timing(h: int):
    """(ms[6], counts[6]) per kernel class: molecules, field pass, plane sample, plane fold,
    molecular current, gather."""
    ms = np.zeros(6)
    cnt = np.zeros(6, np.int64)
    _check(load().ml_timing(C.c_void_p(h), C.c_void_p(_ptr(ms)), C.c_void_p(_ptr(cnt))))
    return ms, cnt


def ml_launch_count(h: int) -> int:
    return int(load().ml_launch_count(C.c_void_p(h)))


def ml_adjoint_run(h: int, nsteps: int, ckpt_every: int, plane: int, freq: int, grad_eps_ptr: int = 0,
                   grad_gamma_ptr: int = 0, on_device: bool = False, stream: int = 0) -> float:
    """Objective (flux of `plane` at frequency index `freq` over nsteps steps) and its
    gradients written to the given buffers (0 = skip)."""
    obj = C.c_double(0.0)
    _check(load().ml_adjoint_run(C.c_void_p(h), int(nsteps), int(ckpt_every), int(plane), int(freq),
                                 C.byref(obj), C.c_void_p(grad_eps_ptr or None), C.c_void_p(grad_gamma_ptr or None),
                                 1 if on_device else 0, C.c_void_p(stream)))
    return float(obj.value)


def ml_set_design_eps(h: int, eps_ptr: int, on_device: bool = False, stream: int = 0):
    _check(load().ml_set_design_eps(C.c_void_p(h), C.c_void_p(eps_ptr), 1 if on_device else 0, C.c_void_p(stream)))


def ml_set_couplings(h: int, gamma_ptr: int, on_device: bool = False, stream: int = 0):
    _check(load().ml_set_couplings(C.c_void_p(h), C.c_void_p(gamma_ptr), 1 if on_device else 0, C.c_void_p(stream)))


def ml_cavity_create(desc: ml_cavity_desc, mdesc: ml_molecule_desc) -> int:
    out = C.c_void_p()
    _check(load().ml_cavity_create(C.byref(desc), C.byref(mdesc), C.byref(out)))
    return out.value


def ml_cavity_destroy(c: int):
    _check(load().ml_cavity_destroy(C.c_void_p(c)))


def ml_cavity_step(c: int, nsteps: int, stream: int = 0):
    _check(load().ml_cavity_step(C.c_void_p(c), int(nsteps), C.c_void_p(stream)))


def ml_cavity_mode(c: int, stream: int = 0) -> np.ndarray:
    out = np.zeros(6)
    _check(load().ml_cavity_mode(C.c_void_p(c), out.ctypes.data_as(C.c_void_p), C.c_void_p(stream)))
    return out


def ml_cavity_get_molecules(c: int, what: int, dst_ptr: int, stream: int = 0):
    _check(load().ml_cavity_get_molecules(C.c_void_p(c), int(what), C.c_void_p(dst_ptr), C.c_void_p(stream)))


def ml_cavity_step_count(c: int) -> int:
    return int(load().ml_cavity_step_count(C.c_void_p(c)))


def ml_drive_create(desc: ml_drive_desc, mdesc: ml_molecule_desc) -> int:
    out = C.c_void_p()
    _check(load().ml_drive_create(C.byref(desc), C.byref(mdesc), C.byref(out)))
    return out.value


def ml_drive_destroy(d: int):
    _check(load().ml_drive_destroy(C.c_void_p(d)))


def ml_drive_step(d: int, nsteps: int, stream: int = 0):
    _check(load().ml_drive_step(C.c_void_p(d), int(nsteps), C.c_void_p(stream)))


def ml_drive_get_molecules(d: int, what: int, dst_ptr: int, stream: int = 0):
    _check(load().ml_drive_get_molecules(C.c_void_p(d), int(what), C.c_void_p(dst_ptr), C.c_void_p(stream)))


def ml_drive_step_count(d: int) -> int:
    return int(load().ml_drive_step_count(C.c_void_p(d)))


def ml_batch_create(handles) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    out = C.c_void_p()
    _check(load().ml_batch_create(arr, len(handles), C.byref(out)))
    return out.value


def ml_batch_step(b: int, nsteps: int, stream: int = 0):
    _check(load().ml_batch_step(C.c_void_p(b), int(nsteps), C.c_void_p(stream)))


def ml_batch_set_tuning(b: int, blocks_per_sm: int, use_graph: bool = True):
    _check(load().ml_batch_set_tuning(C.c_void_p(b), int(blocks_per_sm), 1 if use_graph else 0))


def ml_batch_autotune(b: int, trial_steps: int, stream: int = 0):
    choice = C.c_int(0)
    ms = C.c_double(0.0)
    _check(load().ml_batch_autotune(C.c_void_p(b), int(trial_steps), C.c_void_p(stream), C.byref(choice),
                                    C.byref(ms)))
    return choice.value, ms.value


def ml_batch_launch_count(b: int) -> int:
    return int(load().ml_batch_launch_count(C.c_void_p(b)))


def ml_batch_set_timing(b: int, enable: bool):
    _check(load().ml_batch_set_timing(C.c_void_p(b), int(enable)))


def ml_batch_timing(b: int):
    """(ms[6], counts[6]) per kernel class of the batch's traced launches."""
    ms = np.zeros(6)
    cnt = np.zeros(6, np.int64)
    _check(load().ml_batch_timing(C.c_void_p(b), C.c_void_p(_ptr(ms)), C.c_void_p(_ptr(cnt))))
    return ms, cnt


def ml_batch_destroy(b: int):
    _check(load().ml_batch_destroy(C.c_void_p(b)))


def ml_gather_static(E_ptr: int, nx: int, ny: int, nz: int, periodic, nmol: int, pos_ptr: int,
                     sigma_ptr: int, gamma_ptr: int, out_ptr: int, stream: int = 0):
    """Allocation-free regularised field from a caller-owned FP32 field (device
    pointers; see the header).  Allocates nothing here either: the periodic flags
    travel as a ctypes array on the host."""
    per = (C.c_int * 3)(*[1 if p else 0 for p in periodic])
    _check(load().ml_gather_static(C.c_void_p(E_ptr), nx, ny, nz, per, nmol, C.c_void_p(pos_ptr),
                                   C.c_void_p(sigma_ptr), C.c_void_p(gamma_ptr), C.c_void_p(out_ptr),
                                   C.c_void_p(stream)))


# ---------------------------------------------------------------- Problem wrapper

def grid_desc(prob, precision: int = ML_F32):
    """Marshal a workloads.Problem into ml_grid_desc (plus the arrays it points to)."""
    keep = []
    d = ml_grid_desc()
    d.nx, d.ny, d.nz = prob.nx, prob.ny, prob.nz
    d.courant = prob.courant
    d.precision = precision
    for a in range(3):
        d.periodic[a] = 1 if prob.periodic[a] else 0
    for f in range(6):
        d.pml[f] = prob.pml[f]
    d.pml_m, d.pml_sigma_max = prob.pml_m, prob.pml_sigma_max
    d.pml_kappa_max, d.pml_alpha_max = prob.pml_kappa_max, prob.pml_alpha_max
    d.zchunk = prob.zchunk
    if prob.mat is not None:
        m = np.ascontiguousarray(prob.mat, np.uint8)
        keep.append(m)
        d.mat = _ptr(m)
    mats = (ml_material * len(prob.materials))(*[_material(x) for x in prob.materials])
    keep.append(mats)
    d.n_materials = len(prob.materials)
    d.materials = mats
    if prob.design_box is not None:
        for q in range(6):
            d.design_box[q] = prob.design_box[q]
        de = np.ascontiguousarray(prob.design_eps, np.float64)
        keep.append(de)
        d.design_eps = _ptr(de)
    if prob.sources:
        srcs = (ml_source * len(prob.sources))(*[ml_source(s.axis, s.index, s.comp, s.amp, s.omega, s.width, s.t0)
                                                 for s in prob.sources])
        keep.append(srcs)
        d.n_sources = len(prob.sources)
        d.sources = srcs
    return d, keep


def molecule_desc(mol):
    keep = []

    def arr(x, dt):
        a = np.ascontiguousarray(x, dt)
        keep.append(a)
        return _ptr(a)

    d = ml_molecule_desc()
    d.count = mol.count
    d.nlev = arr(mol.nlev, np.int32)
    d.off = arr(mol.off, np.int64)
    d.pos = arr(mol.pos, np.float64)
    d.sigma = arr(mol.sigma, np.float64)
    d.gamma = arr(mol.gamma, np.float64)
    d.decay = arr(mol.decay, np.float64)
    d.dephase = arr(mol.dephase, np.float64)
    d.kind = arr(mol.kind, np.int32)
    d.nsub = arr(mol.nsub, np.int32)
    d.H0 = arr(np.ascontiguousarray(mol.H0, np.complex128).view(np.float64), np.float64)
    d.mu = arr(np.ascontiguousarray(mol.mu, np.complex128).view(np.float64), np.float64)
    d.rho = arr(np.ascontiguousarray(mol.rho0, np.complex128).view(np.float64), np.float64)
    d.pool = int(mol.H0.shape[0])
    return d, keep


class Cavity:
    """Single-mode cavity (polarisations x, y) coupled to a `workloads.Molecules` table."""

    def __init__(self, molecules, omega_c: float, coupling: float, dt: float, q0=(0.0, 0.0), p0=(0.0, 0.0),
                 precision: int = ML_F32, stream: int = 0):
        d = ml_cavity_desc()
        d.omega_c, d.coupling, d.dt, d.precision = float(omega_c), float(coupling), float(dt), int(precision)
        for l in range(2):
            d.q0[l] = float(q0[l])
            d.p0[l] = float(p0[l])
        md, self._keep = molecule_desc(molecules)
        self.mol = molecules
        self.stream = stream
        self.h = ml_cavity_create(d, md)

    def step(self, n: int = 1):
        ml_cavity_step(self.h, n, self.stream)

    def mode(self) -> np.ndarray:
        """q_x, q_y, p_x, p_y, d_x, d_y."""
        return ml_cavity_mode(self.h, self.stream)

    def molecules(self, what: int) -> np.ndarray:
        M = self.mol.count
        if what == ML_MOL_RHO:
            out = np.zeros(2 * int((self.mol.nlev.astype(np.int64) ** 2).sum()))
            ml_cavity_get_molecules(self.h, what, _ptr(out), self.stream)
            return out.view(np.complex128)
        n = {ML_MOL_EFIELD: 3 * M, ML_MOL_MUDOT: 3 * M, ML_MOL_ENERGY: M, ML_MOL_POP: ML_MAX_LEVELS * M}[what]
        out = np.zeros(n)
        ml_cavity_get_molecules(self.h, what, _ptr(out), self.stream)
        if what in (ML_MOL_EFIELD, ML_MOL_MUDOT):
            return out.reshape(M, 3)
        if what == ML_MOL_POP:
            return out.reshape(M, ML_MAX_LEVELS)
        return out

    def rho(self, m: int) -> np.ndarray:
        n = int(self.mol.nlev[m])
        pool = self.molecules(ML_MOL_RHO)
        off = int(np.concatenate([[0], np.cumsum(self.mol.nlev.astype(np.int64) ** 2)])[m])
        return pool[off:off + n * n].reshape(n, n)

    @property
    def nstep(self) -> int:
        return ml_cavity_step_count(self.h)

    def close(self):
        if self.h:
            ml_cavity_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Drive:
    """Molecules of a `workloads.Molecules` table driven by the prescribed wave of
    Eq. E_analytical (no back-action); positions give each molecule's z."""

    def __init__(self, molecules, amplitude: float, omega: float, phase: float, center: float, half_width: float,
                 polarization, dt: float, precision: int = ML_F32, stream: int = 0):
        d = ml_drive_desc()
        d.amplitude, d.omega, d.phase, d.center = float(amplitude), float(omega), float(phase), float(center)
        d.half_width, d.dt, d.precision = float(half_width), float(dt), int(precision)
        for c in range(3):
            d.polarization[c] = float(polarization[c])
        md, self._keep = molecule_desc(molecules)
        self.mol = molecules
        self.stream = stream
        self.h = ml_drive_create(d, md)

    def step(self, n: int = 1):
        ml_drive_step(self.h, n, self.stream)

    def molecules(self, what: int) -> np.ndarray:
        M = self.mol.count
        if what == ML_MOL_RHO:
            out = np.zeros(2 * int((self.mol.nlev.astype(np.int64) ** 2).sum()))
            ml_drive_get_molecules(self.h, what, _ptr(out), self.stream)
            return out.view(np.complex128)
        n = {ML_MOL_EFIELD: 3 * M, ML_MOL_MUDOT: 3 * M, ML_MOL_ENERGY: M, ML_MOL_POP: ML_MAX_LEVELS * M}[what]
        out = np.zeros(n)
        ml_drive_get_molecules(self.h, what, _ptr(out), self.stream)
        if what in (ML_MOL_EFIELD, ML_MOL_MUDOT):
            return out.reshape(M, 3)
        if what == ML_MOL_POP:
            return out.reshape(M, ML_MAX_LEVELS)
        return out

    def rho(self, m: int) -> np.ndarray:
        n = int(self.mol.nlev[m])
        pool = self.molecules(ML_MOL_RHO)
        off = int(np.concatenate([[0], np.cumsum(self.mol.nlev.astype(np.int64) ** 2)])[m])
        return pool[off:off + n * n].reshape(n, n)

    @property
    def nstep(self) -> int:
        return ml_drive_step_count(self.h)

    def close(self):
        if self.h:
            ml_drive_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several Grids advanced together (one launch per kernel class per step)."""

    def __init__(self, grids, stream: int = 0):
        self.grids = list(grids)
        self.stream = stream
        self.h = ml_batch_create([g.h for g in self.grids])

    def step(self, n: int):
        ml_batch_step(self.h, n, self.stream)

    def tune(self, blocks_per_sm: int, use_graph: bool = True):
        ml_batch_set_tuning(self.h, blocks_per_sm, use_graph)

    def autotune(self, trial_steps: int = 64):
        return ml_batch_autotune(self.h, trial_steps, self.stream)

    @property
    def launches(self) -> int:
        return ml_batch_launch_count(self.h)

    def close(self):
        if getattr(self, "h", None):
            ml_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid:
    """A grid handle built from a Problem (fields, molecules, flux planes)."""

    def __init__(self, prob, precision: int = ML_F32, stream: int = 0, molecules: bool = True):
        self.prob = prob
        self.precision = precision
        self.dtype = np.float64 if precision == ML_F64 else np.float32
        self.stream = stream
        d, keep = grid_desc(prob, precision)
        self.h = ml_grid_create(d, stream)
        try:
            self.planes = []
            for p in prob.planes:
                self.planes.append(ml_add_flux_plane(self.h, p.axis, p.index, p.omegas))
            if molecules and prob.molecules.count:
                md, keep2 = molecule_desc(prob.molecules)
                ml_add_molecules(self.h, md, stream)
        except Exception:
            ml_grid_destroy(self.h)
            self.h = None
            raise

    def close(self):
        if getattr(self, "h", None):
            ml_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.prob.nz, self.prob.ny, self.prob.nx)

    def step(self, n: int = 1):
        ml_step(self.h, n, self.stream)

    def sync(self):
        ml_sync_status(self.h, self.stream)

    @property
    def nstep(self) -> int:
        return ml_step_count(self.h)

    def fields(self, mask: int = ML_ALL) -> List[np.ndarray]:
        ncomp = bin(mask).count("1")
        out = np.zeros((ncomp,) + self.shape, self.dtype)
        ml_get_fields(self.h, mask, _ptr(out), False, self.stream)
        return [out[q] for q in range(ncomp)]

    def set_fields(self, f: List[np.ndarray], mask: int = ML_ALL):
        buf = np.ascontiguousarray(np.stack([np.asarray(x, self.dtype) for x in f]))
        ml_set_fields(self.h, mask, _ptr(buf), False, self.stream)

    def molecules(self, what: int) -> np.ndarray:
        M = self.prob.molecules.count
        if what == ML_MOL_RHO:
            out = np.zeros(2 * int(self.prob.molecules.H0.shape[0]))
            ml_get_molecules(self.h, what, _ptr(out), False, self.stream)
            return out.view(np.complex128)
        n = {ML_MOL_EFIELD: 3 * M, ML_MOL_MUDOT: 3 * M, ML_MOL_ENERGY: M, ML_MOL_POP: ML_MAX_LEVELS * M}[what]
        out = np.zeros(n)
        ml_get_molecules(self.h, what, _ptr(out), False, self.stream)
        if what in (ML_MOL_EFIELD, ML_MOL_MUDOT):
            return out.reshape(M, 3)
        if what == ML_MOL_POP:
            return out.reshape(M, ML_MAX_LEVELS)
        return out

    def rho(self, m: int) -> np.ndarray:
        pool = self.molecules(ML_MOL_RHO)
        mol = self.prob.molecules
        n = int(mol.nlev[m])
        o = int(mol.off[m])
        return pool[o:o + n * n].reshape(n, n)

    def flux(self, p: int) -> np.ndarray:
        return ml_flux(self.h, self.planes[p], len(self.prob.planes[p].omegas), self.stream)

    def plane_data(self, p: int):
        pl = self.prob.planes[p]
        dims = [self.prob.nx, self.prob.ny, self.prob.nz]
        nb, nc = dims[(pl.axis + 1) % 3], dims[(pl.axis + 2) % 3]
        nf = len(pl.omegas)
        z = ml_flux_data(self.h, self.planes[p], 4 * nf * nb * nc, self.stream)
        cnt = nf * nb * nc
        return [z[q * cnt:(q + 1) * cnt].reshape(nf, nc, nb) for q in range(4)]

    def absorbed(self) -> float:
        return ml_absorbed(self.h, self.stream)

    def adjoint(self, nsteps: int, plane: int, freq: int, ckpt_every: int = 100):
        """Flux of `plane` at frequency index `freq` over the next nsteps steps and its
        gradients: (objective, d/d design eps (sz, sy, sx) or None, d/d gamma (nmol))."""
        ge = None
        if self.prob.design_box is not None:
            sx, sy, sz = self.prob.design_box[3:]
            ge = np.zeros((sz, sy, sx))
        gg = np.zeros(max(self.prob.molecules.count, 1))
        obj = ml_adjoint_run(self.h, nsteps, ckpt_every, plane, freq, _ptr(ge) if ge is not None else 0,
                             _ptr(gg), False, self.stream)
        return obj, ge, gg[:self.prob.molecules.count]

    def set_design_eps(self, eps: np.ndarray):
        e = np.ascontiguousarray(eps, np.float64)
        ml_set_design_eps(self.h, _ptr(e), False, self.stream)

    def set_couplings(self, gamma: np.ndarray):
        gm = np.ascontiguousarray(gamma, np.float64)
        ml_set_couplings(self.h, _ptr(gm), False, self.stream)

    def checkpoint(self) -> bytes:
        return ml_checkpoint(self.h, self.stream)

    def restore(self, blob: bytes):
        ml_restore(self.h, blob, self.stream)
