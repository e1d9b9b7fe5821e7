"""The oracle's per-column path on every host core, for parity checks on large samples.

Worker processes are spawned (never forked: the parent may already hold a CUDA context), import
only numpy, the seeded workloads and the oracle, and return slim per-column records, so that a
sample of a few thousand columns of a 10^6-atom system stays cheap to ship back.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _worker(args):
    workload, cols, mu = args
    from oracle import pipeline
    out = []
    for c in pipeline.columns(workload, cols):
        r, rE = pipeline.rho_column(c, mu, workload.kT)
        out.append((c.j, c.pattern, r, rE, c.nu_eff, c.eps, c.c, c.g, len(c.atoms)))
    return out


def rho_columns(workload, cols, mu, processes=None):
    """Oracle columns at a given mu: {j: (pattern, rho (len,4), rhoE (len,4), nu_eff, eps, c, g,
    cluster atoms)}, computed by `processes` spawned workers (default: every host core)."""
    cols = np.asarray(cols)
    n = max(1, min(processes or os.cpu_count() or 1, len(cols)))
    chunks = [cols[i::n] for i in range(n)]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            parts = pool.map(_worker, [(workload, c, mu) for c in chunks])
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {int(rec[0]): rec[1:] for part in parts for rec in part}


def block_ids(row_ptr, col_idx, j, pattern):
    """Pattern blocks e = (I, J) of column j = 4 J + alpha, one per pattern atom I."""
    J = int(j) // 4
    out = np.empty(len(pattern), dtype=np.int64)
    for p, I in enumerate(pattern):
        lo, hi = int(row_ptr[I]), int(row_ptr[I + 1])
        e = lo + int(np.searchsorted(col_idx[lo:hi], J))
        assert e < hi and col_idx[e] == J
        out[p] = e
    return out
