"""COHP / ICOHP and their sigma / pi parts (oracle; test infrastructure only).

Eq. 4 defines C_IJ(e) = -(1/pi) sum_ab H_(J,b);(I,a) Im G_(I,a);(J,b)(e + i0) and Eq. 5 its
Fermi-weighted integral B_IJ. With the density matrix of Eq. 2 this integral is

    B_IJ = sum_ab H_(J,b);(I,a) rho_(I,a);(J,b),

and Eq. 6 states that sum_IJ B_IJ is the electronic (band) energy. For s/p orbitals the off-site
Hamiltonian splits into sigma and pi parts (Eqs. 7-8); in the Slater-Koster table the pi part is
the V_pp_pi (delta_ik - u_i u_k) term of the p-p block, everything else off-site is sigma:

    B^pi_IJ = sum over p-p orbital pairs of V_pp_pi (delta_ik - u_i u_k) rho,  B^sigma = B - B^pi.

On-site pairs (I = J) carry no sigma / pi split; their B_II is part of the sum rule.
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
