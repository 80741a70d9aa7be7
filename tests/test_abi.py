"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(ml_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["ml_grid_create", "ml_add_molecules", "ml_step", "ml_get_fields", "ml_flux"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2512_06173_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2512_06173_gb300 import maxlink
    missing = [n for n in declared_symbols() if not hasattr(maxlink, n)]
    assert not missing, missing


def test_version_and_error_strings():
    from paper_2512_06173_gb300 import maxlink
    lib = maxlink.load()
    assert b"sm_103a" in lib.ml_version()
    assert lib.ml_last_error() is not None


def test_invalid_arguments_are_rejected_without_a_gpu():
    """Argument validation happens before any CUDA call."""
    from paper_2512_06173_gb300 import maxlink
    from paper_2512_06173_gb300.workloads import Material, Problem
    d, keep = maxlink.grid_desc(Problem(8, 8, 8, 0.5))
    d.nx = 0
    with pytest.raises(maxlink.MaxlinkError) as e:
        maxlink.ml_grid_create(d)
    assert e.value.status == maxlink.ML_ERR_INVALID_ARG
    d, keep = maxlink.grid_desc(Problem(8, 8, 8, 0.5, periodic=(True, False, False), pml=(2, 2, 0, 0, 0, 0)))
    with pytest.raises(maxlink.MaxlinkError) as e:
        maxlink.ml_grid_create(d)
    assert "periodic" in str(e.value)
    d, keep = maxlink.grid_desc(Problem(8, 8, 8, 1.5))
    with pytest.raises(maxlink.MaxlinkError):
        maxlink.ml_grid_create(d)
    # pole tables: too many poles, a negative resonance in an extra pole
    d, keep = maxlink.grid_desc(Problem(8, 8, 8, 0.5, materials=[Material(1.0, 0.5, 0.1)]))
    d.materials[0].n_extra = maxlink.ML_MAX_POLES
    with pytest.raises(maxlink.MaxlinkError) as e:
        maxlink.ml_grid_create(d)
    assert e.value.status == maxlink.ML_ERR_INVALID_ARG
    d, keep = maxlink.grid_desc(Problem(8, 8, 8, 0.5, materials=[Material(1.0, 0.5, 0.1, extra=((0.3, 0.1, -0.2),))]))
    with pytest.raises(maxlink.MaxlinkError) as e:
        maxlink.ml_grid_create(d)
    assert "omega0" in str(e.value)
    d, keep = maxlink.grid_desc(Problem(8, 8, 8, 0.5, zchunk=1))
    with pytest.raises(maxlink.MaxlinkError) as e:
        maxlink.ml_grid_create(d)
    assert "zchunk" in str(e.value)
