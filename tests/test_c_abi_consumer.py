"""A plain C program (tests/c_abi/energy_force.c) uses the library through include/elses.h
alone: the header compiles as C99, and on a GPU the program's energy + force evaluation gives the
Python binding's results bit for bit (the binding only marshals arguments)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi", "energy_force.c")
PKG = os.path.join(ROOT, "paper_1210_1531_gb300")


def _cuda_home():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            return cand
    return None


def _cc():
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda = _cuda_home()
    if not cc or not cuda:
        pytest.skip("no C compiler or CUDA headers")
    return cc, cuda


def test_header_compiles_as_c99():
    cc, cuda = _cc()
    res = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", os.path.join(ROOT, "include"),
                          "-I", os.path.join(cuda, "include"), SRC], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr


@pytest.mark.gpu
def test_c_program_matches_the_binding(tmp_path):
    import torch
    import workloads as wl
    from tests import gpu_util as gu
    eg = gu.library()
    cc, cuda = _cc()
    exe = str(tmp_path / "energy_force")
    lib64 = os.path.join(cuda, "lib64")
    res = subprocess.run([cc, "-std=c99", "-O2", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(cuda, "include"),
                          SRC, "-o", exe, "-L", PKG, "-lelses", "-L", lib64, "-lcudart",
                          "-Wl,-rpath," + PKG, "-Wl,-rpath," + lib64], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    w = wl.make("diamond_64")
    sk = eg.make_sk(w.sk)
    params = eg.make_params(w.r_cluster, w.nu, w.kT, w.n_electrons, nu_classes=w.nu_classes)
    inp, out = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(inp, "wb") as f:
        f.write(np.int32(w.n_atoms).tobytes())
        f.write(np.asarray(w.box, dtype=np.float64).tobytes())
        f.write(bytes(sk))
        f.write(bytes(params))
        f.write(np.ascontiguousarray(w.pos, dtype=np.float64).tobytes())
    res = subprocess.run([exe, str(inp), str(out)], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    data = np.fromfile(out, dtype=np.float64)
    mu, e_band, f_free, F = data[0], data[1], data[2], data[3:].reshape(w.n_atoms, 3)
    s = eg.system_for(w)
    mu_p, e_p, f_p, F_p = s.energy_force()
    assert mu == mu_p and e_band == e_p and f_free == f_p
    assert np.array_equal(F, gu.to_np(F_p))
