"""The C-ABI library loads and exports every entry point include/elses.h declares (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "elses.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_1210_1531_gb300 import build
    return build.build()


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|void|const char\*)\s+(elses_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for required in ("elses_build_clusters", "elses_green_columns", "elses_density_matrix",
                     "elses_find_mu", "elses_energy_force"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(elses_\w+)$", out, re.M))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    import paper_1210_1531_gb300 as eg
    assert sorted(eg.EXPORTS) == declared()
    L = eg.load_library(libpath)
    for name in declared():
        assert hasattr(L, name)


def test_loads_without_gpu_and_reports_version(libpath):
    L = ctypes.CDLL(libpath)
    L.elses_version.restype = ctypes.c_int
    assert L.elses_version() == 1
    L.elses_last_error.restype = ctypes.c_char_p
    assert isinstance(L.elses_last_error(), bytes)
    # argument checks happen before any device call
    L.elses_build_clusters.restype = ctypes.c_int
    assert L.elses_build_clusters(None, 0, None, None, None, None, None) == -1
