"""Dense and block-sparse H, S from the Slater-Koster blocks (oracle; test infrastructure only).

H and S are the M x M LCAO matrices of Eq. 1 (M = 4 N for s/p orbitals); basis index
i = 4 I + alpha with orbital alpha in (s, px, py, pz). Block (I, J) holds
H[(I,a),(J,b)] for a, b = 0..3 and is the Slater-Koster block at d = R_J - R_I (minimum image)
when I != J and |d| <= r_cut, the on-site block when I == J, and zero otherwise.
"""
from __future__ import annotations

import numpy as np

from . import slater_koster as skm
from .structure import min_image, neighbor_csr


def pair_vectors(pos, box, row_ptr, col_idx):
    """d = min_image(R_J - R_I) for every block (I, J) of a CSR pattern."""
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    return min_image(pos[col_idx] - pos[rows], box), rows


def bsr_values(pos, box, sk, row_ptr, col_idx):
    """H and S block values (nnzb, 4, 4) on a CSR pattern over all atoms."""
    d, rows = pair_vectors(pos, box, row_ptr, col_idx)
    diag = rows == col_idx
    Hb = np.zeros((len(col_idx), 4, 4))
    Sb = np.zeros((len(col_idx), 4, 4))
    if np.any(~diag):
        h, s = skm.blocks(d[~diag], sk)
        Hb[~diag] = h
        Sb[~diag] = s
    h0, s0 = skm.onsite(sk)
    Hb[diag] = h0
    Sb[diag] = s0
    return Hb, Sb


def dense(pos, box, sk, r_cut=None):
    """Dense H, S (M x M) of a whole (small) system."""
    r_cut = sk.r_cut if r_cut is None else r_cut
    row_ptr, col_idx = neighbor_csr(pos, box, r_cut)
    Hb, Sb = bsr_values(pos, box, sk, row_ptr, col_idx)
    return bsr_to_dense(row_ptr, col_idx, Hb), bsr_to_dense(row_ptr, col_idx, Sb)


def bsr_to_dense(row_ptr, col_idx, vals):
    n = len(row_ptr) - 1
    A = np.zeros((4 * n, 4 * n))
    for I in range(n):
        for e in range(row_ptr[I], row_ptr[I + 1]):
            J = col_idx[e]
            A[4 * I:4 * I + 4, 4 * J:4 * J + 4] = vals[e]
    return A


def bsr_submatrix(row_ptr, col_idx, vals, atoms):
    """Principal submatrix of a block-sparse matrix on the orbitals of `atoms` (sorted list),
    rows/columns ordered by (atom position in `atoms`, orbital); blocks outside the pattern are 0."""
    atoms = np.asarray(atoms)
    n = len(atoms)
    A = np.zeros((n, 4, n, 4))
    for a, I in enumerate(atoms):
        row = col_idx[row_ptr[I]:row_ptr[I + 1]]
        hit = np.searchsorted(atoms, row)
        ok = (hit < n) & (atoms[np.minimum(hit, n - 1)] == row)
        for k in np.nonzero(ok)[0]:
            A[a, :, hit[k], :] = vals[row_ptr[I] + k]
    return A.reshape(4 * n, 4 * n)


def cluster_matrices(pos, box, sk, atoms):
    """Principal submatrices H_C, S_C of H and S on the orbitals of `atoms` (sorted list).

    Rows/columns ordered by (atom position in `atoms`, orbital). Pairs are taken with the
    minimum-image vector between the two atoms, exactly as in the global H and S.
    """
    atoms = np.asarray(atoms)
    p = pos[atoms]
    d = min_image(p[None, :, :] - p[:, None, :], box)       # d[a, b] = R_b - R_a
    r2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]
    a_idx, b_idx = np.nonzero(r2 <= sk.r_cut * sk.r_cut)
    off = a_idx != b_idx
    n = len(atoms)
    Hc = np.zeros((n, 4, n, 4))
    Sc = np.zeros((n, 4, n, 4))
    if np.any(off):
        hb, sb = skm.blocks(d[a_idx[off], b_idx[off]], sk)
        Hc[a_idx[off], :, b_idx[off], :] = hb
        Sc[a_idx[off], :, b_idx[off], :] = sb
    h0, s0 = skm.onsite(sk)
    idx = np.arange(n)
    Hc[idx, :, idx, :] = h0
    Sc[idx, :, idx, :] = s0
    return Hc.reshape(4 * n, 4 * n), Sc.reshape(4 * n, 4 * n)
