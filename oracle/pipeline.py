"""The whole per-column path over a workload (oracle; test infrastructure only).

Order of the memory-saving workflow of Eq. 3: (H, S) => G => mu => (2nd calc. of G) => rho.
Here the per-column quantities needed for the second step are kept instead of recomputed (the
paper states that the workflow choice does not change the resulting physical quantities):

  1. per column j = 4 J + alpha: cluster of atom J, H_C and S_C, Krylov build, projection,
     projected eigenproblem, spectra (e, c, d, g) and the pattern rows of U;
  2. mu by bisection on N(mu) = sum_j sum_k 2 f d c (needs every column) or a given mu;
  3. rho and rhoE columns on the pattern rows P(j) (atoms within r_cut of J):
         rho_(I,b),j = 2 sum_k f_k Z_(I,b),k c_k  with Z = U V;
  4. E_band, Omega, F_free and the forces.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import hamiltonian, krylov, physics
from .structure import cluster, neighbor_csr, transpose_map, within


@dataclasses.dataclass
class Column:
    j: int
    atoms: np.ndarray        # cluster atoms (sorted)
    pattern: np.ndarray      # atoms within r_cut of J (sorted) = pattern rows P(j)
    nu_eff: int
    eps: np.ndarray
    c: np.ndarray
    d: np.ndarray
    g: np.ndarray
    UP: np.ndarray           # U on the pattern rows: (4 * len(pattern), nu_eff)
    V: np.ndarray
    Hp: np.ndarray
    Sp: np.ndarray


def nu_for(workload, n_cluster_atoms):
    """Krylov dimension of a column: the workload's nu, or its size class when it has classes."""
    for (max_atoms, nu) in workload.nu_classes:
        if n_cluster_atoms <= max_atoms:
            return nu
    return workload.nu


def solve_column(pos, box, sk, r_cluster, nu, j, nu_rule=None):
    J, alpha = divmod(int(j), 4)
    atoms = cluster(pos, box, J, r_cluster)
    if nu_rule is not None:
        nu = nu_rule(len(atoms))
    Hc, Sc = hamiltonian.cluster_matrices(pos, box, sk, atoms)
    aJ = int(np.searchsorted(atoms, J))
    jl = 4 * aJ + alpha
    kc = krylov.arnoldi_column(Hc, Sc, jl, nu)
    eps, V = krylov.projected_eig(kc.Hp, kc.Sp)
    c, d, g = krylov.spectra(kc, V, jl)
    pattern = within(pos, box, J, sk.r_cut)
    rows = (4 * np.searchsorted(atoms, pattern)[:, None] + np.arange(4)[None, :]).ravel()
    return Column(int(j), atoms, pattern, kc.nu_eff, eps, c, d, g, kc.U[rows, :], V,
                  kc.Hp, kc.Sp)


def solve_column_matrices(Hc, Sc, atoms, pattern, j, nu):
    """The same per-column path on given cluster matrices (caller values on a caller pattern):
    Hc, Sc are the principal submatrices of H and S on the orbitals of `atoms` (sorted), and the
    pattern rows P(j) are the atoms `pattern` (the caller pattern's row J), inside the cluster."""
    J, alpha = divmod(int(j), 4)
    atoms = np.asarray(atoms)
    jl = 4 * int(np.searchsorted(atoms, J)) + alpha
    kc = krylov.arnoldi_column(Hc, Sc, jl, nu)
    eps, V = krylov.projected_eig(kc.Hp, kc.Sp)
    c, d, g = krylov.spectra(kc, V, jl)
    pattern = np.asarray(pattern)
    rows = (4 * np.searchsorted(atoms, pattern)[:, None] + np.arange(4)[None, :]).ravel()
    return Column(int(j), atoms, pattern, kc.nu_eff, eps, c, d, g, kc.U[rows, :], V, kc.Hp, kc.Sp)


def columns(workload, cols=None):
    """Per-column results for the given basis indices (default: all 4N)."""
    M = 4 * workload.n_atoms
    cols = np.arange(M) if cols is None else np.asarray(cols)
    rule = (lambda n: nu_for(workload, n)) if workload.nu_classes else None
    return [solve_column(workload.pos, workload.box, workload.sk, workload.r_cluster,
                         workload.nu, j, rule) for j in cols]


def rho_column(col: Column, mu, kT):
    """rho and rhoE of one column on its pattern rows, shape (len(pattern), 4) each."""
    f2 = 2.0 * physics.fermi(col.eps, mu, kT)
    Z = col.UP @ col.V
    rho = Z @ (f2 * col.c)
    rhoE = Z @ (f2 * col.eps * col.c)
    return rho.reshape(-1, 4), rhoE.reshape(-1, 4)


def chemical_potential(cols, n_electrons, kT):
    eps = np.concatenate([c.eps for c in cols])
    w = np.concatenate([c.d * c.c for c in cols])
    return physics.bisect_mu(eps, w, n_electrons, kT)


def scalars(cols, mu, kT, n_electrons):
    """N(mu), E_band, Omega and F_free summed over the given columns."""
    N = E = Om = 0.0
    for c in cols:
        f2 = 2.0 * physics.fermi(c.eps, mu, kT)
        N += float(np.sum(f2 * c.d * c.c))
        E += float(np.sum(f2 * c.g * c.c))
        Om += float(np.sum(c.d * c.c * physics.omega(c.eps, mu, kT)))
    return dict(N=N, E_band=E, Omega=Om, F_free=Om + mu * n_electrons)


def assemble(workload, cols, mu):
    """rho and rhoE on the BSR pattern (rho[e][a][b] = rho_(I,a),(J,b) for e = (I, J))."""
    row_ptr, col_idx = neighbor_csr(workload.pos, workload.box, workload.sk.r_cut)
    tmap = transpose_map(row_ptr, col_idx)
    rho = np.zeros((len(col_idx), 4, 4))
    rhoE = np.zeros((len(col_idx), 4, 4))
    for c in cols:
        J, alpha = divmod(c.j, 4)
        r, rE = rho_column(c, mu, workload.kT)
        for p, I in enumerate(c.pattern):
            # block (J, I) sits in row J; its transpose (I, J) holds column j's entries
            e_JI = row_ptr[J] + int(np.searchsorted(col_idx[row_ptr[J]:row_ptr[J + 1]], I))
            e = tmap[e_JI]
            rho[e, :, alpha] = r[p]
            rhoE[e, :, alpha] = rE[p]
    return row_ptr, col_idx, rho, rhoE


def run(workload, mu=None):
    """Whole path on every column: spectra, mu, rho, rhoE, energies and forces."""
    cols = columns(workload)
    iters = None
    if mu is None:
        mu, iters = chemical_potential(cols, workload.n_electrons, workload.kT)
    row_ptr, col_idx, rho, rhoE = assemble(workload, cols, mu)
    F = physics.forces(workload.pos, workload.box, workload.sk, row_ptr, col_idx, rho, rhoE)
    out = dict(mu=mu, bisect_iters=iters, row_ptr=row_ptr, col_idx=col_idx, rho=rho,
               rhoE=rhoE, forces=F, columns=cols)
    out.update(scalars(cols, mu, workload.kT, workload.n_electrons))
    return out


def dense_reference(workload):
    """Exact diagonalisation of the whole system (the plain definition; small systems)."""
    from . import exact
    H, S = hamiltonian.dense(workload.pos, workload.box, workload.sk)
    e, Y = exact.generalized_eig(H, S)
    mu = exact.chemical_potential(e, workload.n_electrons, workload.kT)
    rho, rhoE = exact.density_matrices(e, Y, mu, workload.kT)
    return dict(H=H, S=S, eps=e, Y=Y, mu=mu, rho=rho, rhoE=rhoE,
                E_band=exact.band_energy(e, mu, workload.kT),
                Omega=exact.grand_potential(e, mu, workload.kT))
