"""Seeded random disordered-carbon systems, small enough for the oracle to solve every column:
ragged cluster sizes (slots of 16 and 32 atoms partly filled), several Krylov dimensions and size
classes, both column forms (half-warp and whole-warp), both schedules and both second-pass forms.
Every column's rho is compared with the oracle at the GPU's mu, and mu is checked as a root of
the oracle's N."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import hamiltonian, pipeline, structure
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

# (cells, density g/cm^3, sigma A, seed, r_cluster A, nu, size classes, library options)
CASES = [
    ((2, 2, 2), 3.0, 0.25, 11, 0.0, 24, (), dict(schedule=1)),
    ((2, 2, 2), 3.0, 0.25, 11, 0.0, 24, (), dict(schedule=1, reorth=1)),
    ((3, 3, 3), 2.6, 0.30, 12, 4.0, 12, (), dict()),
    ((3, 3, 3), 2.6, 0.30, 12, 4.0, 12, (), dict(k3_lanes=32, reorth=1)),
    ((3, 3, 3), 3.2, 0.30, 13, 5.0, 20, ((85, 12), (1 << 30, 20)), dict(schedule=1, reorth=1)),
    ((3, 3, 3), 3.2, 0.30, 13, 5.0, 20, ((85, 12), (1 << 30, 20)), dict(schedule=1, autotune=True)),
]


@pytest.fixture(scope="module")
def eg():
    return gu.library()


def _system(cells, density, sigma, seed, r_cl, nu, classes):
    pos, box = wl.amorphous(ncell=cells, density_gcc=density, sigma=sigma, dmin=1.3, seed=seed)
    return wl.Workload(f"amorphous_{np.prod(cells) * 8}_{seed}", pos, box, wl.sk_params(),
                       r_cluster=r_cl, nu=nu, nu_classes=classes)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_every_column_against_the_oracle(eg, case):
    cells, density, sigma, seed, r_cl, nu, classes, opts = CASES[case]
    w = _system(cells, density, sigma, seed, r_cl, nu, classes)
    rp, ci = structure.neighbor_csr(w.pos, w.box, w.sk.r_cut)
    _, S = hamiltonian.bsr_values(w.pos, w.box, w.sk, rp, ci)
    assert np.linalg.eigvalsh(hamiltonian.bsr_to_dense(rp, ci, S)).min() > 0.05   # Eq. 1's S
    s = eg.system_for(w, **opts)
    mu, e_band, _, F = s.energy_force()
    rho, rhoE = s.density_matrix(mu)
    grp, gci = (gu.to_np(t) for t in s.pattern())
    assert np.array_equal(grp, rp) and np.array_equal(gci, ci)
    cols = pipeline.columns(w)
    assert abs(pipeline.scalars(cols, mu, w.kT, w.n_electrons)["N"] - w.n_electrons) < 1e-8
    _, _, rho_o, rhoE_o = pipeline.assemble(w, cols, mu)
    assert np.abs(gu.to_np(rho) - rho_o).max() <= gu.RHO_TOL
    assert np.abs(gu.to_np(rhoE) - rhoE_o).max() <= gu.RHOE_TOL
    sc = pipeline.scalars(cols, mu, w.kT, w.n_electrons)
    assert abs(e_band - sc["E_band"]) / w.n_atoms <= gu.E_TOL_PER_ATOM
    nu_g = gu.to_np(s.spectra()["nu_eff"])
    assert np.array_equal(nu_g, np.array([c.nu_eff for c in cols]))
    assert np.abs(gu.to_np(F).sum(axis=0)).max() < 1e-9


@pytest.mark.parametrize("reorth", [0, 1])
def test_exact_gradient_against_the_oracle(eg, reorth):
    """The exact gradient of the truncated method (dOmega/dH, dOmega/dS on the pattern) on a
    random 64-atom system with nu = 12, every column, against the oracle's autodiff."""
    from oracle import adjoint
    w = _system((2, 2, 2), 3.0, 0.25, 14, 0.0, 12, ())
    s = eg.system_for(w, reorth=reorth)
    mu, _, _, _ = s.energy_force()
    dH, dS = (gu.to_np(t) for t in s.omega_gradient(mu))
    _, _, oH, oS, _ = adjoint.pattern_gradient(w, mu)
    assert np.abs(dH - oH).max() <= 1e-9 * np.abs(oH).max()
    assert np.abs(dS - oS).max() <= 1e-9 * np.abs(oS).max()
