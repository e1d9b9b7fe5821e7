"""Per-column Krylov build, projection and projected eigenproblem (oracle; test only).

The paper solves Eq. 1 column by column with the multiple Arnoldi method and defers its details
to the method's own paper, which is not available. The reading implemented here (the same one
the CUDA path implements) is a Galerkin projection of Eq. 1 onto the Krylov space
K_nu(H_C, e_j) of the cluster matrices, with a basis orthonormal in the S inner product:

    u_1 = e_j / sqrt(S_jj)
    for n = 1 .. nu:
        HU[:, n] = H_C u_n ;  SU[:, n] = S_C u_n
        stop if n = nu
        w = HU[:, n]
        two classical Gram-Schmidt passes in the S inner product:
            h = SU[:, 1..n]^T w ;  w = w - U[:, 1..n] h
        Sw = S_C w ;  beta = sqrt(w^T Sw)
        if w^T Sw < -(1e-12 * ||HU[:, n]||_2)^2 : S is not positive definite (error)
        if beta <= 1e-12 * ||HU[:, n]||_2 : stop (invariant subspace, nu_eff = n)
        u_{n+1} = w / beta
    H' = U^T HU,  S' = U^T SU, each symmetrised as (X + X^T)/2

The projected problem H' v = e S' v is solved as the generalized eigenproblem of Eq. 1's text
(H y = e S y) with the computed S' (not assumed to be I):

    S' = L L^T,  A = L^-1 H' L^-T = Q diag(e) Q^T,  V = L^-T Q,  e ascending.

With Z = U V the Green's function column is G_ij(z) ~ sum_k Z_ik c_k / (z - e_k) where
c = V^T U^T e_j; the spectra kept per column are (e, c, d = V^T (SU)_j, g = V^T (HU)_j), from
which N(mu), E_band and Omega follow (see physics).
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.linalg import solve_triangular

BREAKDOWN_TOL = 1e-12


class NotPositiveDefinite(RuntimeError):
    """S is not positive definite, against the premise of Eq. 1: a Krylov vector w has
    w^T S w < 0 beyond rounding, or the projected overlap S' failed its Cholesky factorisation."""


@dataclasses.dataclass
class KrylovColumn:
    U: np.ndarray      # (n_c, nu_eff) S-orthonormal basis
    SU: np.ndarray     # S_C U
    HU: np.ndarray     # H_C U
    Hp: np.ndarray     # projected H (nu_eff x nu_eff)
    Sp: np.ndarray     # projected S
    nu_eff: int


def arnoldi_column(Hc, Sc, jl, nu, breakdown_tol=BREAKDOWN_TOL):
    """The Krylov build of column `jl` (local index in the cluster), step by step as above."""
    nc = Hc.shape[0]
    U = np.zeros((nc, nu))
    SU = np.zeros((nc, nu))
    HU = np.zeros((nc, nu))
    U[jl, 0] = 1.0 / np.sqrt(Sc[jl, jl])
    nu_eff = nu
    for n in range(nu):
        HU[:, n] = Hc @ U[:, n]
        SU[:, n] = Sc @ U[:, n]
        if n == nu - 1:
            break
        w = HU[:, n].copy()
        for _ in range(2):
            h = SU[:, :n + 1].T @ w
            w = w - U[:, :n + 1] @ h
        Sw = Sc @ w
        wSw = float(w @ Sw)
        hnorm = np.linalg.norm(HU[:, n])
        if wSw < -(breakdown_tol * hnorm) ** 2:
            raise NotPositiveDefinite(f"w^T S w = {wSw:.3e} < 0 at Krylov step {n + 1}")
        beta = np.sqrt(max(wSw, 0.0))
        if beta <= breakdown_tol * hnorm:
            nu_eff = n + 1
            break
        U[:, n + 1] = w / beta
    U, SU, HU = U[:, :nu_eff], SU[:, :nu_eff], HU[:, :nu_eff]
    Hp = U.T @ HU
    Sp = U.T @ SU
    return KrylovColumn(U, SU, HU, 0.5 * (Hp + Hp.T), 0.5 * (Sp + Sp.T), nu_eff)


def projected_eig(Hp, Sp):
    """Solve H' v = e S' v: returns (e ascending, V with V^T S' V = I)."""
    try:
        L = np.linalg.cholesky(Sp)
    except np.linalg.LinAlgError as exc:
        raise NotPositiveDefinite(str(exc)) from exc
    X = solve_triangular(L, Hp, lower=True)
    A = solve_triangular(L, X.T, lower=True).T
    A = 0.5 * (A + A.T)
    e, Q = np.linalg.eigh(A)
    V = solve_triangular(L.T, Q, lower=False)
    return e, V


def spectra(kc: KrylovColumn, V, jl):
    """c = V^T U^T e_j,  d = V^T (SU)^T e_j,  g = V^T (HU)^T e_j."""
    return V.T @ kc.U[jl, :], V.T @ kc.SU[jl, :], V.T @ kc.HU[jl, :]
