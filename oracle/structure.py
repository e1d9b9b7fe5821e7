"""Neighbour lists, clusters and the block-sparse pattern by brute force (oracle; test only).

H and S are sparse because the two-centre integrals vanish beyond r_cut (Eq. 1 and the text on
the LCAO matrices); each column j only touches the local cluster around its atom, which is what
makes the method order-N. Readings:

  * periodic orthorhombic box, minimum-image convention (needs box > 2 r in every direction);
  * the pattern of H and S is every atom pair with |d| <= r_cut, self included, rows sorted;
  * the cluster of atom J is every atom with |d| <= r_cluster (inclusive), J included, sorted;
    r_cluster <= 0 means the whole system.

The distance test is written so that each floating-point operation is a single IEEE operation
in a fixed order (d - box*rint(d/box), then (dx*dx + dy*dy) + dz*dz compared with rc*rc);
that makes the integer outputs reproducible bit for bit by any implementation that performs the
same operations.
"""
from __future__ import annotations

import numpy as np


def min_image(d, box):
    """Minimum-image separation vectors (elementwise IEEE ops: d - box * rint(d / box))."""
    return d - box * np.rint(d / box)


def dist2(d):
    """Squared length as (dx*dx + dy*dy) + dz*dz."""
    return d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]


def within(pos, box, i, r):
    """Sorted indices of atoms within distance r of atom i (inclusive, i itself included)."""
    d = min_image(pos - pos[i], box)
    return np.nonzero(dist2(d) <= r * r)[0]


def neighbor_csr(pos, box, r_cut, rows=None):
    """CSR of neighbour atoms within r_cut (self included). Returns (row_ptr int32, col_idx int32).

    With `rows` given, only those rows are built (row_ptr then refers to that subset, in order).
    """
    pos = np.asarray(pos, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    if np.any(box <= 2.0 * r_cut):
        raise ValueError("box must exceed 2*r_cut in every direction for the minimum image")
    rows = np.arange(len(pos)) if rows is None else np.asarray(rows)
    cols = [within(pos, box, int(i), r_cut) for i in rows]
    row_ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(c) for c in cols])
    col_idx = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    return row_ptr.astype(np.int32), col_idx.astype(np.int32)


def cluster(pos, box, J, r_cluster):
    """Atoms of the cluster of atom J (sorted ascending). r_cluster <= 0: the whole system."""
    if r_cluster <= 0.0:
        return np.arange(len(pos))
    box = np.asarray(box, dtype=np.float64)
    if np.any(box <= 2.0 * r_cluster):
        raise ValueError("box must exceed 2*r_cluster in every direction for the minimum image")
    return within(pos, box, J, r_cluster)


def transpose_map(row_ptr, col_idx):
    """For every block e = (I, J), the index of block (J, I) in the same (symmetric) pattern."""
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    key = {(int(i), int(j)): e for e, (i, j) in enumerate(zip(rows, col_idx))}
    return np.array([key[(int(j), int(i))] for i, j in zip(rows, col_idx)], dtype=np.int64)
