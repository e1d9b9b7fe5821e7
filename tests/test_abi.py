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


def _header_fields(struct):
    """(name, C type, array length) of the members of `struct` in include/elses.h, in order."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (struct, struct), text, re.S).group(1)
    out = []
    for decl in filter(None, (d.strip() for d in body.split(";"))):
        m = re.match(r"(long long|double|int)\s+(.*)$", decl, re.S)
        assert m, decl
        for item in m.group(2).split(","):
            a = re.match(r"\s*(\w+)\s*(?:\[(\d+)\])?\s*$", item)
            out.append((a.group(1), m.group(1), int(a.group(2)) if a.group(2) else 0))
    return out


@pytest.mark.parametrize("struct, cls", [("elses_sk", "SK"), ("elses_params", "Params"),
                                         ("elses_stats", "Stats")])
def test_binding_structs_match_the_header(struct, cls):
    """The ctypes mirrors of the header's structs have the same members, types and order."""
    import paper_1210_1531_gb300 as eg
    ctype = {"double": ctypes.c_double, "int": ctypes.c_int, "long long": ctypes.c_longlong}
    want = []
    for name, t, n in _header_fields(struct):
        want.append((name, ctype[t] * n if n else ctype[t]))
    got = getattr(eg, cls)._fields_
    assert [n for n, _ in got] == [n for n, _ in want]
    for (n, a), (_, b) in zip(got, want):
        assert ctypes.sizeof(a) == ctypes.sizeof(b) and getattr(a, "_type_", a) == getattr(b, "_type_", b), n


BAD_PARAMS = [("nu", 0, "nu must be"), ("nu", 65, "nu must be"), ("n_classes", 5, "n_classes"),
              ("kT", 0.0, "kT must be positive"), ("force_mode", 2, "force_mode"),
              ("krylov_block", 2, "krylov_block"), ("batch_atoms", -1, "batch_atoms"),
              ("k3_lanes", 16, "k3_lanes"), ("max_qr_sweeps", -1, "max_qr_sweeps"),
              ("reorth", 2, "reorth"), ("keep_factors", -1, "keep_factors"),
              ("r_cluster", 1.0, "r_cluster must be >= r_cut")]


@pytest.mark.parametrize("field, value, message", BAD_PARAMS, ids=[f"{f}={v}" for f, v, _ in BAD_PARAMS])
def test_build_rejects_bad_parameters_before_any_device_call(libpath, field, value, message):
    """elses_build_clusters checks every parameter on the host before it touches the device or
    the positions (here a host buffer stands in for the device pointer): ELSES_ERR_ARG and a
    message naming the parameter, no system created."""
    import paper_1210_1531_gb300 as eg
    import workloads as wl
    w = wl.make("diamond_64")
    p = eg.make_params(6.0, w.nu, w.kT, w.n_electrons)
    setattr(p, field, value)
    L = eg.load_library(libpath)
    L.elses_last_error.restype = ctypes.c_char_p
    sk = eg.make_sk(w.sk)
    box = (ctypes.c_double * 3)(20.0, 20.0, 20.0)
    pos = (ctypes.c_double * (3 * w.n_atoms))()
    h = ctypes.c_void_p(None)
    rc = L.elses_build_clusters(ctypes.byref(h), w.n_atoms, ctypes.cast(pos, ctypes.c_void_p), box,
                                ctypes.byref(sk), ctypes.byref(p), None)
    assert rc == -1 and h.value is None
    assert message in L.elses_last_error().decode()
