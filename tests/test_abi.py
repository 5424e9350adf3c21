"""The C-ABI library loads and exports every entry point include/fsi.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "fsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(fsi_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ["fsi_create_mesh", "fsi_init_phases", "fsi_residual", "fsi_jvp", "fsi_gmres", "fsi_step"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2402_10348_gb300 import _build, fsi
    _build.build()
    lib = ctypes.CDLL(fsi.LIB_PATH)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(fsi.EXPORTS) == declared()
