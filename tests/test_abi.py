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


def test_header_is_plain_c_and_the_binding_matches_its_layouts(tmp_path):
    """include/maxlink.h compiles as C99 with warnings as errors, and every descriptor
    struct the binding mirrors has the same size and field offsets in C and in ctypes."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2512_06173_gb300 import maxlink
    structs = {"ml_pole": maxlink.ml_pole, "ml_material": maxlink.ml_material, "ml_source": maxlink.ml_source,
               "ml_grid_desc": maxlink.ml_grid_desc, "ml_molecule_desc": maxlink.ml_molecule_desc,
               "ml_cavity_desc": maxlink.ml_cavity_desc, "ml_drive_desc": maxlink.ml_drive_desc}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "maxlink.h"', "int main(void) {"]
    for s, cls in structs.items():
        lines.append(f'    printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in cls._fields_:
            lines.append(f'    printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                         check=True).stdout.splitlines())
    for s, cls in structs.items():
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, f"{s}.{f}"
