"""Fermi-Dirac occupation, chemical-potential bisection, energies and forces (oracle; test only).

Eq. 2 defines rho_ij = -(1/pi) Int f(e - mu) Im G_ij(e + i0) de with the Fermi-Dirac occupation
f and chemical potential mu; with G_ij(z) = sum_k Z_ik c_k / (z - e_k) (poles e_k, residues
Z_ik c_k) the integral is done by residues: Im 1/(e + i0 - e_k) = -pi delta(e - e_k), so

    rho_ij   = 2 sum_k f(e_k - mu) Z_ik c_k           (factor 2: spin; reading of the text)
    rhoE_ij  = 2 sum_k f(e_k - mu) e_k Z_ik c_k        (energy-weighted density matrix)
    N(mu)    = Tr(rho S) = sum_j sum_k 2 f(e_k - mu) d_k c_k
    E_band   = Tr(rho H) = sum_j sum_k 2 f(e_k - mu) g_k c_k        (= sum of ICOHP, Eq. 6)
    Omega    = sum_j sum_k d_k c_k w(e_k),   w(e) = -2 kT ln(1 + exp(-(e - mu)/kT))
    F_free   = Omega + mu N_e

mu is found by bisection on N(mu) = N_e once G has been computed the first time (Eq. 3 and
the text after it). The bisection reading: bracket [min e - 40 kT, max e + 40 kT] over all poles; at
each step mid = (lo + hi)/2 replaces lo if N(mid) < N_e, else hi; stop when hi - lo < 1e-13 eV
or after 100 steps; mu = (lo + hi)/2. No sign change on the bracket is an error.

Forces: the gradient of F_free at fixed N_e equals that of Omega at fixed mu, and
dOmega/dH_ji = rho_ij, dOmega/dS_ji = -rhoE_ij (exact when the Krylov space spans the
cluster, as for exact diagonalisation).
"""
from __future__ import annotations

import numpy as np

from . import slater_koster as skm
from .hamiltonian import pair_vectors


class NoBracket(RuntimeError):
    """N(mu) - N_e has no sign change on the bisection bracket."""


def fermi(eps, mu, kT):
    """f(e - mu) = 1 / (1 + exp((e - mu)/kT)), evaluated without overflow."""
    x = (np.asarray(eps, dtype=np.float64) - mu) / kT
    out = np.empty_like(x)
    p = x > 0
    e = np.exp(-x[p])
    out[p] = e / (1.0 + e)
    out[~p] = 1.0 / (1.0 + np.exp(x[~p]))
    return out


def omega(eps, mu, kT):
    """Grand-potential weight w(e) = -2 kT ln(1 + exp(-(e - mu)/kT)); dw/de = 2 f."""
    x = (np.asarray(eps, dtype=np.float64) - mu) / kT
    out = np.empty_like(x)
    p = x >= 0
    out[p] = -2.0 * kT * np.log1p(np.exp(-x[p]))
    out[~p] = 2.0 * (x[~p] * kT) - 2.0 * kT * np.log1p(np.exp(x[~p]))
    return out


def electron_count(eps, w, mu, kT):
    """N(mu) = sum 2 f(e - mu) w over poles e with weights w = d c."""
    return float(np.sum(2.0 * fermi(eps, mu, kT) * w))


def bisect_mu(eps, w, n_electrons, kT, tol=1e-13, max_iter=100):
    """Chemical potential by bisection (reading in the module docstring). Returns (mu, iters)."""
    eps = np.asarray(eps, dtype=np.float64).ravel()
    w = np.asarray(w, dtype=np.float64).ravel()
    lo = float(eps.min()) - 40.0 * kT
    hi = float(eps.max()) + 40.0 * kT
    if not (electron_count(eps, w, lo, kT) < n_electrons <= electron_count(eps, w, hi, kT)):
        raise NoBracket("electron count not bracketed")
    it = 0
    while it < max_iter and hi - lo >= tol:
        mid = 0.5 * (lo + hi)
        if electron_count(eps, w, mid, kT) < n_electrons:
            lo = mid
        else:
            hi = mid
        it += 1
    return 0.5 * (lo + hi), it


def forces(pos, box, sk, row_ptr, col_idx, rho, rhoE):
    """F_K = -sum_ij [rho_ij dH_ji/dR_K - rhoE_ij dS_ji/dR_K] on a symmetric BSR pattern.

    rho[e][a][b] = rho_(I,a),(J,b) for block e = (I, J). H is symmetric, so each block pairs
    with the same-position block of dH. Block (I, J) depends on d = R_J - R_I only.
    """
    d, rows = pair_vectors(pos, box, row_ptr, col_idx)
    off = rows != col_idx
    gH, gS = skm.block_grads(d[off], sk)
    g = (np.einsum("pab,pmab->pm", rho[off], gH) - np.einsum("pab,pmab->pm", rhoE[off], gS))
    F = np.zeros((len(pos), 3))
    np.add.at(F, col_idx[off], -g)
    np.add.at(F, rows[off], g)
    return F
