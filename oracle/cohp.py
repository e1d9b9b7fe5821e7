"""COHP / ICOHP and their sigma / pi parts (oracle; test infrastructure only).

Eq. 4 defines C_IJ(e) = -(1/pi) sum_ab H_(J,b);(I,a) Im G_(I,a);(J,b)(e + i0) and Eq. 5 its
Fermi-weighted integral B_IJ. With the density matrix of Eq. 2 this integral is

    B_IJ = sum_ab H_(J,b);(I,a) rho_(I,a);(J,b),

and Eq. 6 states that sum_IJ B_IJ is the electronic (band) energy. For s/p orbitals the off-site
Hamiltonian splits into sigma and pi parts (Eqs. 7-8); in the Slater-Koster table the pi part is
the V_pp_pi (delta_ik - u_i u_k) term of the p-p block, everything else off-site is sigma:

    B^pi_IJ = sum over p-p orbital pairs of V_pp_pi (delta_ik - u_i u_k) rho,  B^sigma = B - B^pi.

On-site pairs (I = J) carry no sigma / pi split; their B_II is part of the sum rule.

Energy-resolved: C_IJ at complex energies z = e + i eta (a Lorentzian of width eta in place of
the delta functions of Im G(e + i0)), from G on the pattern, and the density of states
-(1/pi) Im Tr(G S) from the pole weights of N(mu).
"""
from __future__ import annotations

import numpy as np

from . import slater_koster as skm
from .hamiltonian import bsr_values, pair_vectors


def icohp(pos, box, sk, row_ptr, col_idx, rho):
    """(B, B_sigma, B_pi) per block e = (I, J) of the pattern (B_sigma = B_pi = 0 on-site)."""
    Hb, _ = bsr_values(pos, box, sk, row_ptr, col_idx)
    # H symmetric: H_(J,b);(I,a) = H_(I,a);(J,b) = Hb[e][a][b]
    B = np.einsum("eab,eab->e", Hb, rho)
    d, rows = pair_vectors(pos, box, row_ptr, col_idx)
    off = rows != col_idx
    Bpi = np.zeros(len(col_idx))
    if np.any(off):
        dd = d[off]
        r = np.sqrt(np.einsum("pi,pi->p", dd, dd))
        u = dd / r[:, None]
        vppp = skm.radial(r, sk.V0, sk.qH, sk)[:, 3]
        Hpi = vppp[:, None, None] * (np.eye(3)[None] - np.einsum("pi,pk->pik", u, u))
        Bpi[off] = np.einsum("pik,pik->p", Hpi, rho[off][:, 1:, 1:])
    Bsig = np.where(off, B - Bpi, 0.0)
    return B, Bsig, Bpi


def green_pattern(workload, cols, z):
    """G(z) on the pattern for the given columns: complex [nnzb][4][4][n_z] with
    [e][a][b][iz] = G_(I,a),(J,b)(z_iz) for e = (I, J) (the layout of rho), from the poles and
    residues of each column, G_ij(z) = sum_k Z_ik c_k / (z - e_k) (module physics)."""
    from .structure import neighbor_csr, transpose_map
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    row_ptr, col_idx = neighbor_csr(workload.pos, workload.box, workload.sk.r_cut)
    tmap = transpose_map(row_ptr, col_idx)
    G = np.zeros((len(col_idx), 4, 4, len(z)), dtype=np.complex128)
    for c in cols:
        J, alpha = divmod(c.j, 4)
        Zm = c.UP @ c.V
        g = Zm @ (c.c[:, None] / (z[None, :] - c.eps[:, None]))      # [4 |P|][n_z]
        g = g.reshape(len(c.pattern), 4, len(z))
        for p, I in enumerate(c.pattern):
            e_JI = row_ptr[J] + int(np.searchsorted(col_idx[row_ptr[J]:row_ptr[J + 1]], I))
            G[tmap[e_JI], :, alpha, :] = g[p]
    return row_ptr, col_idx, G


def cohp_spectrum(workload, cols, z):
    """Eq. 4 at complex energies z = e + i eta: C_IJ(z) = -(1/pi) Im sum_ab H_(J,b);(I,a)
    G_(I,a);(J,b)(z) per block e = (I, J), and its sigma / pi parts (as for icohp).
    Returns (C, C_sigma, C_pi), each [nnzb][n_z]."""
    row_ptr, col_idx, G = green_pattern(workload, cols, z)
    pos, box, sk = workload.pos, workload.box, workload.sk
    Hb, _ = bsr_values(pos, box, sk, row_ptr, col_idx)
    C = -np.einsum("eab,eabz->ez", Hb, G.imag) / np.pi
    d, rows = pair_vectors(pos, box, row_ptr, col_idx)
    off = rows != col_idx
    Cpi = np.zeros_like(C)
    if np.any(off):
        dd = d[off]
        r = np.sqrt(np.einsum("pi,pi->p", dd, dd))
        u = dd / r[:, None]
        vppp = skm.radial(r, sk.V0, sk.qH, sk)[:, 3]
        Hpi = vppp[:, None, None] * (np.eye(3)[None] - np.einsum("pi,pk->pik", u, u))
        Cpi[off] = -np.einsum("pik,pikz->pz", Hpi, G.imag[off][:, 1:, 1:, :]) / np.pi
    Csig = np.where(off[:, None], C - Cpi, 0.0)
    return C, Csig, Cpi


def dos(cols, z):
    """Density of states -(1/pi) Im Tr(G(z) S) = -(1/pi) Im sum_j sum_k d_k c_k / (z - e_k)
    (the weights of N(mu)) at complex energies z, summed over the given columns."""
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    out = np.zeros(len(z))
    for c in cols:
        out += -np.imag((c.d * c.c)[None, :] / (z[:, None] - c.eps[None, :])).sum(axis=1) / np.pi
    return out
