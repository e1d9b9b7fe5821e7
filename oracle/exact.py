"""Plain definitions on a whole (small) system: the oracle's exact reference (test only).

Eq. 1 is solved instead of the generalized eigenvalue equation H y_k = e_k S y_k; for tiny
systems that equation is solved here directly, giving the exact result the Krylov method must
reproduce when its subspace is complete:

    S = L L^T,  A = L^-1 H L^-T = Q diag(e) Q^T,  y_k = L^-T q_k   (y_k^T S y_l = delta_kl)
    rho  = 2 sum_k f(e_k - mu) y_k y_k^T,   rhoE = 2 sum_k f(e_k - mu) e_k y_k y_k^T
    mu   : 2 sum_k f(e_k - mu) = N_e (same bisection as the Krylov path, unit weights)
    E_band = 2 sum_k f(e_k - mu) e_k,   Omega = sum_k w(e_k)
    G(z) e_j = (z S - H)^-1 e_j by a dense complex solve.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

from . import physics


def generalized_eig(H, S):
    """Eigenpairs of H y = e S y via Cholesky of S; returns (e ascending, Y with Y^T S Y = I)."""
    L = np.linalg.cholesky(S)
    X = solve_triangular(L, H, lower=True)
    A = solve_triangular(L, X.T, lower=True).T
    A = 0.5 * (A + A.T)
    e, Q = np.linalg.eigh(A)
    Y = solve_triangular(L.T, Q, lower=False)
    return e, Y


def chemical_potential(e, n_electrons, kT):
    mu, _ = physics.bisect_mu(e, np.ones_like(e), n_electrons, kT)
    return mu


def density_matrices(e, Y, mu, kT):
    f2 = 2.0 * physics.fermi(e, mu, kT)
    rho = (Y * f2) @ Y.T
    rhoE = (Y * (f2 * e)) @ Y.T
    return rho, rhoE


def band_energy(e, mu, kT):
    return float(np.sum(2.0 * physics.fermi(e, mu, kT) * e))


def grand_potential(e, mu, kT):
    return float(np.sum(physics.omega(e, mu, kT)))


def green_column(H, S, z, j):
    """Column j of G(z) = (z S - H)^-1 by a dense complex solve (Eq. 1 with b = e_j)."""
    b = np.zeros(H.shape[0], dtype=np.complex128)
    b[j] = 1.0
    return np.linalg.solve(z * S - H, b)
