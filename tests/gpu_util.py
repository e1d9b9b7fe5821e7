"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on the same inputs."""
import dataclasses

import numpy as np
import torch

import workloads as wl
from oracle import pipeline, physics, structure

RHO_TOL = 1e-10          # |delta rho_ij| gate against the same-algorithm oracle
E_TOL_PER_ATOM = 1e-9    # |delta E| / atom (eV)
# rhoE = sum_k Z_ik 2 f(e_k) e_k c_k is rho with every pole's term weighted by its energy; the
# poles that f lets through lie within about 20 eV below mu here, so the rho gate is carried over
# in units of 10 eV (1e-9 eV), below the largest weight
RHOE_TOL = 10.0 * RHO_TOL


def mu_tolerance(system, mu, dn=1e-10, h=1e-4):
    """Bound on the distance between two bisection results whose N(mu) differ by rounding: the
    crossing of N_e moves by delta N / N'(mu), so a difference of up to `dn` electrons (far above
    the rounding of N over every pole of these systems, about 1e-11) allows dn / N'(mu), with
    N' from a central difference of the system's own N; plus twice the bisection's resolution
    (each result lies within half a 1e-13 bracket of its crossing). In a gap N is nearly flat
    and the bound widens accordingly; where N is steep it stays near the resolution."""
    slope = (system.energies(mu + h)["N"] - system.energies(mu - h)["N"]) / (2.0 * h)
    return 2e-13 + dn / max(slope, 1e-300)


def library():
    from paper_1210_1531_gb300 import build
    build.build()
    import paper_1210_1531_gb300 as eg
    eg.load_library()
    return eg


def fragment(n_atoms=16, nu=None):
    """Isolated piece of displaced diamond in a 30 A box; cluster = whole (M = 4 n_atoms)."""
    pos, _ = wl.diamond((2, 2, 2), sigma=0.05)
    c = pos.mean(axis=0)
    keep = np.sort(np.argsort(np.linalg.norm(pos - c, axis=1))[:n_atoms])
    p = pos[keep] - c + 15.0
    return wl.Workload(f"fragment_{n_atoms}", p, np.full(3, 30.0), wl.sk_params(), r_cluster=0.0,
                       nu=4 * n_atoms if nu is None else nu)


def to_np(t):
    return t.detach().cpu().numpy()


def rho_of_column(rho, row_ptr, col_idx, j, pattern):
    """Column j of a BSR rho (rho[e][a][b] = rho_(I,a),(J,b)) on the pattern atoms: (len, 4)."""
    J, alpha = divmod(int(j), 4)
    out = np.zeros((len(pattern), 4))
    for p, I in enumerate(pattern):
        row = col_idx[row_ptr[I]:row_ptr[I + 1]]
        e = row_ptr[I] + int(np.searchsorted(row, J))
        assert col_idx[e] == J
        out[p] = rho[e, :, alpha]
    return out


def oracle_rho_columns(workload, cols, mu):
    """Oracle columns at a given mu: {j: (pattern, rho (len,4), rhoE (len,4), column)}."""
    res = {}
    for c in pipeline.columns(workload, cols):
        r, rE = pipeline.rho_column(c, mu, workload.kT)
        res[c.j] = (c.pattern, r, rE, c)
    return res


def max_rho_diff(gpu_rho, gpu_rhoE, row_ptr, col_idx, oracle_cols):
    dr = dE = 0.0
    for j, (pattern, r, rE, _) in oracle_cols.items():
        dr = max(dr, np.abs(rho_of_column(gpu_rho, row_ptr, col_idx, j, pattern) - r).max())
        dE = max(dE, np.abs(rho_of_column(gpu_rhoE, row_ptr, col_idx, j, pattern) - rE).max())
    return dr, dE


def spectral_moments(eps, w, nu, m_max=3):
    """Invariant moments sum_k w_k eps_k^m (m = 0..m_max) of one column's poles."""
    e = eps[:nu]
    return np.array([np.sum(w[:nu] * e ** m) for m in range(m_max + 1)])


def significant_poles_match(eps_g, c_g, eps_o, c_o, tol=1e-9, cmin=1e-6):
    """Poles with a non-negligible residue weight |c_k| > cmin must agree. Poles whose weight is
    at rounding level (e.g. from symmetry-decoupled directions of a perfect lattice, where the
    Krylov space picks up rounding noise) do not enter G, rho or E and are not unique."""
    sig = np.abs(c_o) > cmin
    for e, c in zip(eps_o[sig], c_o[sig]):
        k = int(np.argmin(np.abs(eps_g - e)))
        if abs(eps_g[k] - e) > tol or abs(abs(c_g[k]) - abs(c)) > 1e-7 * max(1.0, abs(c)):
            return False
    return int(np.sum(np.abs(c_g) > 10 * cmin)) <= int(np.sum(sig))


def oracle_electron_count(workload, cols_all, mu):
    return pipeline.scalars(cols_all, mu, workload.kT, workload.n_electrons)["N"]


def with_nu(workload, nu):
    return dataclasses.replace(workload, nu=nu)


__all__ = ["physics", "structure", "torch"]
