"""bench.py's rho check on CPU: the gather plan over the BSR pattern picks the rows of each column
that the oracle returns, the comparison is exact when the arrays agree, and one changed element
of rho or rhoE anywhere in the sampled rows is reported.

The oracle's own rho and rhoE, assembled on the BSR pattern (pipeline.assemble), stand in for
the library's arrays here; on the GPU the same plan indexes the device arrays."""
import numpy as np

import bench
import workloads as wl
from oracle import pipeline


def test_gather_plan_matches_oracle_columns_and_catches_one_element():
    w = wl.make("diamond_64")
    mu = 0.4
    cols = np.array([0, 5, 130, 255])
    row_ptr, col_idx, rho, rhoE = pipeline.assemble(w, pipeline.columns(w), mu)
    v, cores, orc = bench.oracle_columns(w, cols, mu)
    assert sorted(orc) == list(cols) and v > 0 and cores >= 1
    pats, e, b = bench.gather_plan(row_ptr, col_idx, cols)
    gpu = bench.split_columns(cols, pats, rho[e, :, b], rhoE[e, :, b])
    assert bench.compare_rho(gpu, orc) == (0.0, 0.0)
    for arr, which in ((rho, 0), (rhoE, 1)):
        planted = arr.copy()
        planted[e[7], 2, b[7]] += 3e-10                # one element of one sampled row
        g = (planted, rhoE) if which == 0 else (rho, planted)
        gpu = bench.split_columns(cols, pats, g[0][e, :, b], g[1][e, :, b])
        d = bench.compare_rho(gpu, orc)
        assert d[which] > 2.9e-10 and d[1 - which] == 0.0
