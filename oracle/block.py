"""Block Krylov build per atom, one space started by the atom's 4 orbitals (oracle; test only).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The alternative reading of the multiple Arnoldi method (module krylov): the m_orb = 4 orbitals of
atom J start one block Krylov space K(H_C, E_J) = span{E_J, H E_J, H^2 E_J, ...},
E_J = [e_4J, e_4J+1, e_4J+2, e_4J+3], shared by the atom's 4 columns of Eq. 1. Its basis is
orthonormal in the S inner product and is built one vector at a time (the band form of block
Arnoldi, lag b = number of starting vectors):

    u_1 .. u_b: the starting vectors, each taken through two classical Gram-Schmidt passes
                against the ones before it and normalised in the S norm;
    for m = 1, 2, ...:  HU[:, m] = H_C u_m
        while the basis has fewer than nu vectors:
            w = HU[:, m]; two CGS passes in the S inner product against every basis vector so far
            (h = SU^T w, w -= U h); Sw = S_C w; beta = sqrt(w^T Sw);
            w^T Sw < -(1e-12 ||HU[:, m]||_2)^2 means S is not positive definite (error);
            beta <= 1e-12 ||HU[:, m]||_2 ends the extension (nu_eff = the basis size);
            u_{m+b} = w / beta
    and every basis vector u gets SU = S_C u (by a product) when it is made.

With b = 1 this is exactly the per-column build of module krylov. The projected problem
(H' = U^T HU, S' = U^T SU, symmetrised, generalized eigenproblem by module krylov) is solved once
per atom; column j = 4J + alpha keeps its own spectra c = V^T U^T e_j, d = V^T (SU)^T e_j,
g = V^T (HU)^T e_j and pattern rows of U, so everything downstream (bisection, rho, energies,
forces) is the per-column path unchanged. nu is the dimension of the block space (b nu_b after
nu_b block steps).
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian, krylov
from .krylov import BREAKDOWN_TOL, KrylovColumn
from .pipeline import Column
from .structure import cluster, within


def block_arnoldi(Hc, Sc, jls, nu, breakdown_tol=BREAKDOWN_TOL):
    """The band build above for starting columns `jls` (local indices); nu total vectors."""
    nc = Hc.shape[0]
    b = len(jls)
    U = np.zeros((nc, nu))
    SU = np.zeros((nc, nu))
    HU = np.zeros((nc, nu))
    n = 0
    for jl in jls:
        w = np.zeros(nc)
        w[jl] = 1.0
        for _ in range(2):
            h = SU[:, :n].T @ w
            w = w - U[:, :n] @ h
        Sw = Sc @ w
        beta = np.sqrt(max(float(w @ Sw), 0.0))
        if not beta > 0.0:
            raise krylov.NotPositiveDefinite("starting vectors are linearly dependent in the S norm")
        U[:, n] = w / beta
        SU[:, n] = Sc @ U[:, n]
        n += 1
    nu_eff, extend = nu, True
    m = 0
    while m < nu_eff:
        HU[:, m] = Hc @ U[:, m]
        if extend and n < nu:
            w = HU[:, m].copy()
            for _ in range(2):
                h = SU[:, :n].T @ w
                w = w - U[:, :n] @ h
            Sw = Sc @ w
            wSw = float(w @ Sw)
            hnorm = np.linalg.norm(HU[:, m])
            if wSw < -(breakdown_tol * hnorm) ** 2:
                raise krylov.NotPositiveDefinite(f"w^T S w = {wSw:.3e} < 0")
            beta = np.sqrt(max(wSw, 0.0))
            if beta <= breakdown_tol * hnorm:
                extend = False
                nu_eff = n
            else:
                U[:, n] = w / beta
                SU[:, n] = Sc @ U[:, n]
                n += 1
        m += 1
    U, SU, HU = U[:, :nu_eff], SU[:, :nu_eff], HU[:, :nu_eff]
    Hp = U.T @ HU
    Sp = U.T @ SU
    return KrylovColumn(U, SU, HU, 0.5 * (Hp + Hp.T), 0.5 * (Sp + Sp.T), nu_eff)


def solve_atom(pos, box, sk, r_cluster, nu, J):
    """The 4 columns of atom J from one block space: a list of pipeline.Column."""
    atoms = cluster(pos, box, J, r_cluster)
    Hc, Sc = hamiltonian.cluster_matrices(pos, box, sk, atoms)
    aJ = int(np.searchsorted(atoms, J))
    jls = [4 * aJ + a for a in range(4)]
    kc = block_arnoldi(Hc, Sc, jls, nu)
    eps, V = krylov.projected_eig(kc.Hp, kc.Sp)
    pattern = within(pos, box, J, sk.r_cut)
    rows = (4 * np.searchsorted(atoms, pattern)[:, None] + np.arange(4)[None, :]).ravel()
    out = []
    for a, jl in enumerate(jls):
        c, d, g = krylov.spectra(kc, V, jl)
        out.append(Column(4 * J + a, atoms, pattern, kc.nu_eff, eps, c, d, g, kc.U[rows, :], V,
                          kc.Hp, kc.Sp))
    return out


def columns(workload, atoms=None):
    """Columns of the given atoms (default: all), 4 per atom, in column order."""
    atoms = np.arange(workload.n_atoms) if atoms is None else np.asarray(atoms)
    out = []
    for J in atoms:
        out.extend(solve_atom(workload.pos, workload.box, workload.sk, workload.r_cluster,
                              workload.nu, int(J)))
    return out
