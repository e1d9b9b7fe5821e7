"""Exact gradient of the grand potential through the truncated Krylov build (oracle; test only).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The forces of Eq. 2's density matrix use the Hellmann-Feynman adjoint dOmega/dH = rho,
dOmega/dS = -rhoE (module physics). That adjoint is the gradient of Omega only when the Krylov
space spans the cluster; at a truncated nu the space K_nu(H_C, e_j) itself moves with H, and the
gradient of the truncated method has further terms. This module gives that gradient by its plain
definition: the derivative of the same-algorithm column path (module krylov) with respect to the
entries of H_C and S_C, taken by reverse-mode automatic differentiation of a step-for-step
transcription of that path in PyTorch (CPU, float64):

    u_1 = e_j / sqrt(S_jj); CGS2 in the S inner product with S u recomputed by a product;
    breakdown as in krylov.arnoldi_column; H' = U^T HU, S' = U^T SU, each symmetrised;
    S' = L L^T,  A = L^-1 H' L^-T,  p = L^-1 (SU)_j,  q = L^-1 U_j,
    Omega_j = p^T w(A) q,   w(e) = -2 kT ln(1 + exp(-(e - mu)/kT)).

With A = Q diag(e) Q^T the spectra of module krylov are d = Q^T p and c = Q^T q, so Omega_j is
sum_k d_k c_k w(e_k), the column's share of Omega (module physics). The matrix function w(A)
carries its derivative explicitly (Daleckii-Krein): d w(A) = Q (Gamma o (Q^T dA Q)) Q^T with
Gamma_kl the divided difference of w at (e_k, e_l) and Gamma_kk = w'(e_k) = 2 f(e_k).

The gradient of F_free = Omega + mu N_e at fixed N_e equals that of Omega at fixed mu (since
dOmega/dmu = -N(mu) = -N_e at the chemical potential), so the forces are
F_K = -sum_e [dOmega/dH_e : dH_e/dR_K + dOmega/dS_e : dS_e/dR_K] over the pattern blocks e,
the Slater-Koster block derivatives of module slater_koster.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hamiltonian, physics
from .krylov import BREAKDOWN_TOL
from .pipeline import nu_for
from .structure import cluster, neighbor_csr

_F64 = torch.float64


def omega_divided_differences(e, mu, kT):
    """Gamma_kl = (w(e_k) - w(e_l)) / (e_k - e_l), Gamma_kk = w'(e_k) = 2 f(e_k).

    For |e_k - e_l| <= kT the difference is taken in the exact form
    w(a) - w(b) = -2 kT log1p(f(b) expm1(-(a - b)/kT)), free of cancellation.
    """
    e = np.asarray(e, dtype=np.float64)
    w = physics.omega(e, mu, kT)
    f = physics.fermi(e, mu, kT)
    a, b = e[:, None], e[None, :]
    dx = (a - b) / kT
    fb = np.broadcast_to(f[None, :], dx.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        direct = (w[:, None] - w[None, :]) / (a - b)
        near = -2.0 * kT * np.log1p(fb * np.expm1(-dx)) / (a - b)
    G = np.where(np.abs(dx) > 1.0, direct, near)
    same = a == b
    G[same] = np.broadcast_to(2.0 * f[:, None], G.shape)[same]
    return G


class _OmegaOfMatrix(torch.autograd.Function):
    """w(A) = Q diag(w(e)) Q^T for symmetric A, with the Daleckii-Krein derivative."""

    @staticmethod
    def forward(ctx, A, mu, kT):
        e, Q = torch.linalg.eigh(A.detach())
        w = torch.from_numpy(physics.omega(e.numpy(), mu, kT))
        G = torch.from_numpy(omega_divided_differences(e.numpy(), mu, kT))
        ctx.save_for_backward(Q, G)
        return (Q * w[None, :]) @ Q.T

    @staticmethod
    def backward(ctx, grad):
        Q, G = ctx.saved_tensors
        g = 0.5 * (grad + grad.T)
        return Q @ (G * (Q.T @ g @ Q)) @ Q.T, None, None


def column_omega(Hc, Sc, jl, nu, mu, kT, breakdown_tol=BREAKDOWN_TOL):
    """Omega_j of the column with local index jl as a differentiable function of (H_C, S_C)."""
    nc = Hc.shape[0]
    u = torch.zeros(nc, dtype=_F64)
    u[jl] = 1.0
    u = u / torch.sqrt(Sc[jl, jl])
    U, SU, HU = [], [], []
    for n in range(nu):
        U.append(u)
        HU.append(Hc @ u)
        SU.append(Sc @ u)
        if n == nu - 1:
            break
        Um, SUm = torch.stack(U, 1), torch.stack(SU, 1)
        w = HU[n]
        for _ in range(2):
            w = w - Um @ (SUm.T @ w)
        beta = torch.sqrt(torch.clamp(w @ (Sc @ w), min=0.0))
        if float(beta.detach()) <= breakdown_tol * float(torch.linalg.norm(HU[n].detach())):
            break
        u = w / beta
    U, SU, HU = torch.stack(U, 1), torch.stack(SU, 1), torch.stack(HU, 1)
    Hp = U.T @ HU
    Sp = U.T @ SU
    Hp = 0.5 * (Hp + Hp.T)
    Sp = 0.5 * (Sp + Sp.T)
    L = torch.linalg.cholesky(Sp)
    X = torch.linalg.solve_triangular(L, Hp, upper=False)
    A = torch.linalg.solve_triangular(L, X.T, upper=False).T
    A = 0.5 * (A + A.T)
    p = torch.linalg.solve_triangular(L, SU[jl, :, None], upper=False)[:, 0]
    q = torch.linalg.solve_triangular(L, U[jl, :, None], upper=False)[:, 0]
    return p @ (_OmegaOfMatrix.apply(A, mu, kT) @ q)


def column_gradient(Hc, Sc, jl, nu, mu, kT):
    """(Omega_j, dOmega_j/dH_C, dOmega_j/dS_C) for dense numpy cluster matrices."""
    H = torch.tensor(Hc, dtype=_F64, requires_grad=True)
    S = torch.tensor(Sc, dtype=_F64, requires_grad=True)
    om = column_omega(H, S, jl, nu, mu, kT)
    gH, gS = torch.autograd.grad(om, (H, S))
    return float(om.detach()), gH.numpy(), gS.numpy()


def pattern_gradient(workload, mu, cols=None):
    """dOmega/dH and dOmega/dS summed over the given columns (default: all 4N), on the BSR
    pattern of H: arrays [nnzb][4][4] with [e][a][b] = dOmega / dH_(I,a),(J,b) for e = (I, J).
    Also returns the summed Omega of those columns."""
    pos, box, sk = workload.pos, workload.box, workload.sk
    row_ptr, col_idx = neighbor_csr(pos, box, sk.r_cut)
    dH = np.zeros((len(col_idx), 4, 4))
    dS = np.zeros((len(col_idx), 4, 4))
    M = 4 * workload.n_atoms
    cols = np.arange(M) if cols is None else np.asarray(cols)
    omega = 0.0
    for j in cols:
        J, alpha = divmod(int(j), 4)
        atoms = cluster(pos, box, J, workload.r_cluster)
        nu = nu_for(workload, len(atoms)) if workload.nu_classes else workload.nu
        Hc, Sc = hamiltonian.cluster_matrices(pos, box, sk, atoms)
        jl = 4 * int(np.searchsorted(atoms, J)) + alpha
        om, gH, gS = column_gradient(Hc, Sc, jl, nu, mu, workload.kT)
        omega += om
        gH = gH.reshape(len(atoms), 4, len(atoms), 4)
        gS = gS.reshape(len(atoms), 4, len(atoms), 4)
        # the cluster's blocks are the pattern blocks between its atoms
        for a, I in enumerate(atoms):
            row = col_idx[row_ptr[I]:row_ptr[I + 1]]
            hit = np.searchsorted(atoms, row)
            ok = (hit < len(atoms)) & (atoms[np.minimum(hit, len(atoms) - 1)] == row)
            for k in np.nonzero(ok)[0]:
                e = row_ptr[I] + k
                dH[e] += gH[a, :, hit[k], :]
                dS[e] += gS[a, :, hit[k], :]
    return row_ptr, col_idx, dH, dS, omega


def exact_forces(workload, mu, cols=None):
    """F_K = -dOmega/dR_K at fixed mu through the truncated Krylov path (summed columns)."""
    row_ptr, col_idx, dH, dS, _ = pattern_gradient(workload, mu, cols)
    return physics.forces(workload.pos, workload.box, workload.sk, row_ptr, col_idx, dH, -dS)
