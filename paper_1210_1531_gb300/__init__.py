"""GB300 per-column Krylov Green's-function library: Python binding of include/elses.h.

The binding only marshals arguments (ctypes structs, device pointers of torch tensors, the
current CUDA stream) into the C ABI of ``libelses.so``; every step of the method runs in the
library's CUDA kernels. There is no CPU fallback: without the built library (sm_103a) every
call raises.

    sys = System(pos_cuda_f64, box, sk, r_cluster=6.0, nu=30, kT=0.1, n_electrons=4*N)
    mu, e_band, f_free, forces = sys.energy_force()
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libelses.so")

ERRORS = {
    -1: "ELSES_ERR_ARG", -2: "ELSES_ERR_NOT_SPD", -3: "ELSES_ERR_NONFINITE",
    -4: "ELSES_ERR_NO_BRACKET", -5: "ELSES_ERR_TIMEOUT", -6: "ELSES_ERR_CUDA", -7: "ELSES_ERR_OOM",
    -8: "ELSES_ERR_NOT_IMPLEMENTED", -9: "ELSES_ERR_STATE", -10: "ELSES_ERR_CAPACITY",
}
WARN_BREAKDOWN = 1


class ElsesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class SK(ctypes.Structure):
    _fields_ = [("Es", ctypes.c_double), ("Ep", ctypes.c_double),
                ("V0", ctypes.c_double * 4), ("qH", ctypes.c_double * 4),
                ("S0", ctypes.c_double * 4), ("qS", ctypes.c_double * 4),
                ("r0", ctypes.c_double), ("r_on", ctypes.c_double), ("r_cut", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("r_cluster", ctypes.c_double), ("kT", ctypes.c_double),
                ("n_electrons", ctypes.c_double), ("breakdown_tol", ctypes.c_double),
                ("mu_tol", ctypes.c_double), ("nu", ctypes.c_int), ("max_bisect", ctypes.c_int),
                ("two_pass", ctypes.c_int), ("n_classes", ctypes.c_int),
                ("class_max_atoms", ctypes.c_int * 4), ("class_nu", ctypes.c_int * 4),
                ("max_neighbors", ctypes.c_int), ("max_cluster", ctypes.c_int),
                ("schedule", ctypes.c_int), ("timing", ctypes.c_int), ("k3_ctas_per_sm", ctypes.c_int),
                ("force_mode", ctypes.c_int), ("krylov_block", ctypes.c_int),
                ("batch_atoms", ctypes.c_int), ("autotune", ctypes.c_int), ("graph", ctypes.c_int),
                ("k3_lanes", ctypes.c_int), ("max_qr_sweeps", ctypes.c_int),
                ("reorth", ctypes.c_int), ("keep_factors", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("columns", ctypes.c_longlong),
                ("krylov_launches", ctypes.c_longlong), ("bisect_steps", ctypes.c_int),
                ("k3_ctas_per_sm", ctypes.c_int), ("t_krylov_ms", ctypes.c_double),
                ("t_eig_ms", ctypes.c_double), ("t_bisect_ms", ctypes.c_double),
                ("t_density_ms", ctypes.c_double), ("t_force_ms", ctypes.c_double),
                ("krylov_flops", ctypes.c_double), ("t_adjoint_ms", ctypes.c_double),
                ("adjoint_flops", ctypes.c_double), ("kept_rotations", ctypes.c_longlong),
                ("v_formed_columns", ctypes.c_longlong), ("batches", ctypes.c_int),
                ("keep_factors", ctypes.c_int)]


EXPORTS = (
    "elses_build_clusters", "elses_set_hs", "elses_green_columns", "elses_find_mu",
    "elses_density_matrix", "elses_energies", "elses_energy_force", "elses_forces",
    "elses_omega_gradient", "elses_icohp", "elses_cohp_spectrum", "elses_autotune",
    "elses_get_pattern",
    "elses_get_hs", "elses_get_clusters", "elses_get_spectra", "elses_get_stats",
    "elses_reset_stats", "elses_probe_fp64", "elses_find_mu_static", "elses_system_destroy",
    "elses_last_error", "elses_version",
)

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libelses.so (built by paper_1210_1531_gb300.build) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_1210_1531_gb300.build`")
    L = ctypes.CDLL(path)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    pI, pD, pLL = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)
    sig = {
        "elses_build_clusters": [ctypes.POINTER(P), I, P, pD, ctypes.POINTER(SK), ctypes.POINTER(Params), V],
        "elses_set_hs": [P, I, P, P, P, P, V],
        "elses_green_columns": [P, I, I, I, pD, P, P, V],
        "elses_find_mu": [P, pD, pD, V],
        "elses_density_matrix": [P, D, P, P, V],
        "elses_energies": [P, D, pD, pD, pD, pD, V],
        "elses_energy_force": [P, pD, pD, pD, P, V],
        "elses_icohp": [P, P, P, P, P, V],
        "elses_forces": [P, P, V],
        "elses_omega_gradient": [P, D, I, I, P, P, V],
        "elses_cohp_spectrum": [P, I, pD, P, P, P, pD, V],
        "elses_autotune": [P, I, I, pI, pI, V],
        "elses_get_pattern": [P, pI, P, P, V],
        "elses_get_hs": [P, P, P, V],
        "elses_get_clusters": [P, pLL, pI, P, P, V],
        "elses_get_spectra": [P, pI, P, P, P, P, P, V],
        "elses_get_stats": [P, ctypes.POINTER(Stats)],
        "elses_reset_stats": [P],
        "elses_probe_fp64": [pD, V],
        "elses_find_mu_static": [I, I, P, P, P, P, P, D, D, D, I, pD, pD, pD, V],
        "elses_system_destroy": [P],
        "elses_last_error": [],
        "elses_version": [],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = I
    L.elses_system_destroy.restype = None
    L.elses_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc: int) -> int:
    if rc < 0:
        raise ElsesError(rc, load_library().elses_last_error().decode())
    return rc


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_sk(p) -> SK:
    """SK struct from any object with Es, Ep, V0, qH, S0, qS, r0, r_on, r_cut attributes."""
    s = SK()
    s.Es, s.Ep = float(p.Es), float(p.Ep)
    for name in ("V0", "qH", "S0", "qS"):
        arr = getattr(s, name)
        for x, v in enumerate(getattr(p, name)):
            arr[x] = float(v)
    s.r0, s.r_on, s.r_cut = float(p.r0), float(p.r_on), float(p.r_cut)
    return s


def make_params(r_cluster, nu, kT, n_electrons, two_pass=False, nu_classes=(), schedule=0,
                max_neighbors=0, max_cluster=0, breakdown_tol=0.0, mu_tol=0.0,
                max_bisect=0, timing=False, k3_ctas_per_sm=0, exact_forces=False,
                krylov_block=False, batch_atoms=0, autotune=False, graph=False, k3_lanes=0,
                max_qr_sweeps=0, reorth=0, keep_factors=0) -> Params:
    p = Params()
    p.r_cluster, p.kT, p.n_electrons = float(r_cluster), float(kT), float(n_electrons)
    p.breakdown_tol, p.mu_tol = float(breakdown_tol), float(mu_tol)
    p.nu, p.max_bisect, p.two_pass = int(nu), int(max_bisect), int(bool(two_pass))
    p.n_classes = len(nu_classes)
    for c, (max_atoms, cnu) in enumerate(nu_classes):
        p.class_max_atoms[c] = int(min(max_atoms, 2**31 - 1))
        p.class_nu[c] = int(cnu)
    p.max_neighbors, p.max_cluster, p.schedule = int(max_neighbors), int(max_cluster), int(schedule)
    p.timing = int(bool(timing))
    p.k3_ctas_per_sm = int(k3_ctas_per_sm)
    p.force_mode = 1 if exact_forces else 0
    p.krylov_block = 1 if krylov_block else 0
    p.batch_atoms = int(batch_atoms)
    p.autotune = 1 if autotune else 0
    p.graph = 1 if graph else 0
    p.k3_lanes = int(k3_lanes)
    p.max_qr_sweeps = int(max_qr_sweeps)
    p.reorth = int(reorth)
    p.keep_factors = int(keep_factors)
    return p


class System:
    """One atomic system on the current CUDA device (wraps an elses_system handle).

    The keyword arguments map to the fields of elses_params (include/elses.h): the workflow
    (two_pass), the size classes of nu (nu_classes), the Krylov launch form (schedule: 0 plain,
    1 work queue; k3_ctas_per_sm; k3_lanes: 0 automatic half-warp columns, 32 one warp per
    column; autotune: time the launch shapes at build), the step's CUDA-graph replay (graph),
    the forces (exact_forces: the gradient of the truncated method), block-start Krylov spaces
    (krylov_block), the batch size (batch_atoms), the QR sweep cap of the projected eigenproblem
    (max_qr_sweeps, 0: 30 nu), the second Gram-Schmidt pass (reorth: 0 a second classical pass,
    1 its coefficients from the projected overlap S'), the eigen-factors kept across batches
    (keep_factors: 0 never, 1 a pool sized from the free memory, n >= 2 a pool of n rotations
    per column) and per-call
    event timings (timing).
    """

    def __init__(self, pos, box, sk, r_cluster, nu, kT, n_electrons, two_pass=False,
                 nu_classes=(), schedule=0, max_neighbors=0, max_cluster=0, timing=False,
                 k3_ctas_per_sm=0, exact_forces=False, krylov_block=False, batch_atoms=0,
                 autotune=False, graph=False, k3_lanes=0, max_qr_sweeps=0, reorth=0, keep_factors=0,
                 stream=None):
        self._L = load_library()
        self._h = ctypes.c_void_p(None)
        self.n = int(pos.shape[0])
        self.M = 4 * self.n
        self.sk = make_sk(sk)
        self.params = make_params(r_cluster, nu, kT, n_electrons, two_pass, nu_classes, schedule,
                                  max_neighbors, max_cluster, timing=timing,
                                  k3_ctas_per_sm=k3_ctas_per_sm, exact_forces=exact_forces,
                                  krylov_block=krylov_block, batch_atoms=batch_atoms,
                                  autotune=autotune, graph=graph, k3_lanes=k3_lanes,
                                  max_qr_sweeps=max_qr_sweeps, reorth=reorth, keep_factors=keep_factors)
        self.box = (ctypes.c_double * 3)(*[float(b) for b in box])
        self.rebuild(pos, stream)

    def rebuild(self, pos, stream=None):
        """elses_build_clusters for (new) positions: a CUDA float64 tensor [N, 3]."""
        if not (pos.is_cuda and pos.dtype == torch.float64 and pos.shape == (self.n, 3)):
            raise ValueError("pos must be a CUDA float64 tensor of shape [N, 3]")
        self._pos = pos.contiguous()
        _check(self._L.elses_build_clusters(ctypes.byref(self._h), self.n, _ptr(self._pos),
                                            self.box, ctypes.byref(self.sk),
                                            ctypes.byref(self.params), _stream(stream)))
        nnzb = ctypes.c_int(0)
        _check(self._L.elses_get_pattern(self._h, ctypes.byref(nnzb), None, None, _stream(stream)))
        self.nnzb = nnzb.value

    def autotune(self, stream=None):
        """elses_autotune: the Krylov launch shape timed per cluster size class. Returns
        {class capacity in atoms: (resident CTAs per SM, queue order)}, the order "static"
        (plain schedule), "size" or "atom"."""
        return self._shapes(1, stream)

    def autotune_shapes(self, stream=None):
        """The Krylov launch shapes in use, as autotune() returns them."""
        return self._shapes(0, stream)

    def _shapes(self, run, stream):
        out = (ctypes.c_int * 48)()
        n = ctypes.c_int(0)
        _check(self._L.elses_autotune(self._h, run, 16, out, ctypes.byref(n), _stream(stream)))
        names = {0: "static", 1: "size", 2: "atom"}
        return {out[3 * i]: (out[3 * i + 1], names.get(out[3 * i + 2], "?")) for i in range(min(n.value, 16))}

    # ------------------------------------------------------------------ a3-a10
    def green_columns(self, col_begin=0, col_end=None, z=None, stream=None):
        """Krylov columns [col_begin, col_end). With z (complex sequence) returns G on the pattern
        as a complex128 tensor [nnzb, 4, 4, n_z]; otherwise returns the status (0 or warning)."""
        col_end = self.M if col_end is None else col_end
        if z is None:
            return _check(self._L.elses_green_columns(self._h, col_begin, col_end, 0, None, None,
                                                      None, _stream(stream)))
        zs = [complex(v) for v in z]
        zh = (ctypes.c_double * (2 * len(zs)))(*[x for v in zs for x in (v.real, v.imag)])
        G = torch.zeros((self.nnzb, 4, 4, len(zs), 2), dtype=torch.float64, device="cuda")
        _check(self._L.elses_green_columns(self._h, col_begin, col_end, len(zs), zh, _ptr(G), None,
                                           _stream(stream)))
        return torch.view_as_complex(G)

    def find_mu(self, stream=None):
        mu, n = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(self._L.elses_find_mu(self._h, ctypes.byref(mu), ctypes.byref(n), _stream(stream)))
        return mu.value, n.value

    def density_matrix(self, mu, rho=None, rhoE=None, stream=None):
        rho = torch.empty((self.nnzb, 4, 4), dtype=torch.float64, device="cuda") if rho is None else rho
        rhoE = torch.empty_like(rho) if rhoE is None else rhoE
        _check(self._L.elses_density_matrix(self._h, float(mu), _ptr(rho), _ptr(rhoE), _stream(stream)))
        return rho, rhoE

    def energies(self, mu, stream=None):
        out = [ctypes.c_double(0.0) for _ in range(4)]
        _check(self._L.elses_energies(self._h, float(mu), *[ctypes.byref(o) for o in out], _stream(stream)))
        return dict(N=out[0].value, E_band=out[1].value, Omega=out[2].value, F_free=out[3].value)

    def energy_force(self, forces=None, stream=None):
        """Whole path: returns (mu, E_band, F_free, forces [N, 3] CUDA float64)."""
        forces = torch.empty((self.n, 3), dtype=torch.float64, device="cuda") if forces is None else forces
        mu, e, f = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(self._L.elses_energy_force(self._h, ctypes.byref(mu), ctypes.byref(e), ctypes.byref(f),
                                          _ptr(forces), _stream(stream)))
        return mu.value, e.value, f.value, forces

    def forces(self, out=None, stream=None):
        """a10 alone (elses_forces) from the rho of the last energy_force: CUDA float64 [N, 3]."""
        out = torch.empty((self.n, 3), dtype=torch.float64, device="cuda") if out is None else out
        _check(self._L.elses_forces(self._h, _ptr(out), _stream(stream)))
        return out

    def omega_gradient(self, mu, atom_begin=0, atom_end=None, stream=None):
        """Exact dOmega/dH, dOmega/dS at mu through the truncated Krylov method (elses_omega_gradient),
        summed over the columns of atoms [atom_begin, atom_end): CUDA float64 [nnzb, 4, 4] each."""
        atom_end = self.n if atom_end is None else atom_end
        dH = torch.empty((self.nnzb, 4, 4), dtype=torch.float64, device="cuda")
        dS = torch.empty_like(dH)
        _check(self._L.elses_omega_gradient(self._h, float(mu), int(atom_begin), int(atom_end), _ptr(dH),
                                            _ptr(dS), _stream(stream)))
        return dH, dS

    def cohp_spectrum(self, z, sigma_pi=True, stream=None):
        """Energy-resolved COHP per pattern block and the DOS at complex energies z (Eq. 4,
        elses_cohp_spectrum): (C, C_sigma, C_pi) CUDA float64 [nnzb, n_z] (sigma / pi None unless
        requested) and dos, a numpy array [n_z]."""
        zs = [complex(v) for v in z]
        zh = (ctypes.c_double * (2 * len(zs)))(*[x for v in zs for x in (v.real, v.imag)])
        C = torch.empty((self.nnzb, len(zs)), dtype=torch.float64, device="cuda")
        Cs = torch.empty_like(C) if sigma_pi else None
        Cp = torch.empty_like(C) if sigma_pi else None
        dos = (ctypes.c_double * len(zs))()
        _check(self._L.elses_cohp_spectrum(self._h, len(zs), zh, _ptr(C), _ptr(Cs), _ptr(Cp), dos,
                                           _stream(stream)))
        return C, Cs, Cp, np.array(dos[:])

    def icohp(self, rho, stream=None):
        """(pi)COHP integrals per pattern block: (B, B_sigma, B_pi), CUDA float64 [nnzb] each."""
        B = torch.empty(self.nnzb, dtype=torch.float64, device="cuda")
        Bs, Bp = torch.empty_like(B), torch.empty_like(B)
        _check(self._L.elses_icohp(self._h, _ptr(rho.contiguous()), _ptr(B), _ptr(Bs), _ptr(Bp),
                                   _stream(stream)))
        return B, Bs, Bp

    # ------------------------------------------------------------------ accessors (copies)
    def pattern(self, stream=None):
        rp = torch.empty(self.n + 1, dtype=torch.int32, device="cuda")
        ci = torch.empty(self.nnzb, dtype=torch.int32, device="cuda")
        _check(self._L.elses_get_pattern(self._h, None, _ptr(rp), _ptr(ci), _stream(stream)))
        return rp, ci

    def hs(self, stream=None):
        H = torch.empty((self.nnzb, 4, 4), dtype=torch.float64, device="cuda")
        S = torch.empty_like(H)
        _check(self._L.elses_get_hs(self._h, _ptr(H), _ptr(S), _stream(stream)))
        return H, S

    def set_hs(self, H, S, row_ptr=None, col_idx=None, stream=None):
        """elses_set_hs: caller H and S (CUDA float64 [nnzb, 4, 4]) on the system's own pattern,
        or on the caller's block pattern (CUDA int32 row_ptr [N+1] and col_idx [nnzb])."""
        if (row_ptr is None) != (col_idx is None):
            raise ValueError("row_ptr and col_idx go together")
        nnzb = 0
        if row_ptr is not None:
            row_ptr = row_ptr.to(torch.int32).contiguous()
            col_idx = col_idx.to(torch.int32).contiguous()
            nnzb = int(col_idx.numel())
        _check(self._L.elses_set_hs(self._h, nnzb, _ptr(row_ptr), _ptr(col_idx), _ptr(H.contiguous()),
                                    _ptr(S.contiguous()), _stream(stream)))
        if row_ptr is not None:
            self.nnzb = nnzb

    def clusters(self, stream=None):
        total, mx = ctypes.c_longlong(0), ctypes.c_int(0)
        _check(self._L.elses_get_clusters(self._h, ctypes.byref(total), ctypes.byref(mx), None, None,
                                          _stream(stream)))
        if self.params.r_cluster <= 0:
            return None, None, mx.value
        cp = torch.empty(self.n + 1, dtype=torch.int32, device="cuda")
        cidx = torch.empty(max(1, total.value), dtype=torch.int32, device="cuda")
        _check(self._L.elses_get_clusters(self._h, None, None, _ptr(cp), _ptr(cidx), _stream(stream)))
        return cp, cidx[:total.value], mx.value

    def spectra(self, stream=None):
        nm = ctypes.c_int(0)
        _check(self._L.elses_get_spectra(self._h, ctypes.byref(nm), None, None, None, None, None,
                                         _stream(stream)))
        shape = (self.M, nm.value)
        t = {k: torch.empty(shape, dtype=torch.float64, device="cuda") for k in ("eps", "c", "d", "g")}
        nu_eff = torch.empty(self.M, dtype=torch.int32, device="cuda")
        _check(self._L.elses_get_spectra(self._h, None, _ptr(t["eps"]), _ptr(t["c"]), _ptr(t["d"]),
                                         _ptr(t["g"]), _ptr(nu_eff), _stream(stream)))
        t["nu_eff"] = nu_eff
        return t

    def stats(self):
        st = Stats()
        _check(self._L.elses_get_stats(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in Stats._fields_}

    def reset_stats(self):
        _check(self._L.elses_reset_stats(self._h))

    def close(self):
        if self._h:
            self._L.elses_system_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FreeEnergy(torch.autograd.Function):
    """F_free(R) = Omega + mu N_e of a System at positions R, differentiable in R.

    forward: rebuild at R, then the whole path through elses_energy_force without forces;
    backward: the library's adjoint kernels (elses_forces: dF/dH = rho, dF/dS = -rhoE chained
    with dH/dR, dS/dR, or the exact gradient of the truncated method for a System built with
    exact_forces=True), grad_R = -F * grad_out. Returns (F_free, E_band); E_band is not
    differentiable."""

    @staticmethod
    def forward(ctx, pos, system):
        system.rebuild(pos.detach().contiguous())
        mu = ctypes.c_double(0.0)
        e, f = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(system._L.elses_energy_force(system._h, ctypes.byref(mu), ctypes.byref(e),
                                            ctypes.byref(f), None, _stream(None)))
        ctx.system = system
        e_band = pos.new_tensor(e.value)
        ctx.mark_non_differentiable(e_band)
        return pos.new_tensor(f.value), e_band

    @staticmethod
    def backward(ctx, grad_f, grad_e):
        forces = ctx.system.forces()
        return -forces * grad_f, None


def free_energy(pos, system):
    """Differentiable (F_free, E_band) of `system` at CUDA float64 positions `pos` [N, 3]."""
    return FreeEnergy.apply(pos, system)


def probe_fp64(stream=None) -> float:
    """Measured FP64 FMA throughput of the current device, GFLOP/s (elses_probe_fp64)."""
    g = ctypes.c_double(0.0)
    _check(load_library().elses_probe_fp64(ctypes.byref(g), _stream(stream)))
    return g.value


def find_mu_static(eps, c, d, nu_eff, kT, n_electrons, g=None, mu_tol=0.0, max_bisect=0,
                   stream=None):
    """elses_find_mu_static on CUDA tensors eps, c, d (float64 [M, nu_max]) and nu_eff (int32 [M]).

    For callers that cannot allocate device memory: the library side allocates nothing (its
    scratch is a static device array). Returns (mu, N(mu), E_band or None)."""
    M, nm = eps.shape
    mu, n, e = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load_library().elses_find_mu_static(
        int(M), int(nm), _ptr(eps), _ptr(c), _ptr(d), _ptr(g), _ptr(nu_eff), float(kT),
        float(n_electrons), float(mu_tol), int(max_bisect), ctypes.byref(mu), ctypes.byref(n),
        ctypes.byref(e) if g is not None else None, _stream(stream)))
    return mu.value, n.value, (e.value if g is not None else None)


def system_for(workload, stream=None, **kw):
    """System for a workloads.Workload (positions moved to the current CUDA device)."""
    pos = torch.as_tensor(workload.pos, dtype=torch.float64).cuda()
    return System(pos, workload.box, workload.sk, workload.r_cluster, workload.nu, workload.kT,
                  workload.n_electrons, nu_classes=workload.nu_classes, stream=stream, **kw)
