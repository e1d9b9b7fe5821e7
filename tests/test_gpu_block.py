"""Block-start Krylov spaces (krylov_block = 1) on the GPU against the block oracle (oracle.block).

Gates as for the per-column path: |delta rho_ij| <= 1e-10, |delta E|/atom <= 1e-9 eV against the
same-algorithm oracle at the GPU's mu; exact diagonalisation when the block space is the whole
space, to 1e-8.
"""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import block, hamiltonian, pipeline
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eg():
    return gu.library()


def _oracle_cols(workload, atoms, mu):
    out = {}
    for c in block.columns(workload, atoms):
        r, rE = pipeline.rho_column(c, mu, workload.kT)
        out[c.j] = (c.pattern, r, rE, c)
    return out


@pytest.fixture(scope="module")
def d64(eg):
    w = dataclasses.replace(wl.make("diamond_64"), nu=32)      # 8 block steps of 4
    s = eg.system_for(w, krylov_block=True)
    mu, e_band, f_free, _ = s.energy_force()
    rho, rhoE = s.density_matrix(mu)
    rp, ci = s.pattern()
    return dict(w=w, sys=s, mu=mu, e_band=e_band, f_free=f_free, rho=gu.to_np(rho),
                rhoE=gu.to_np(rhoE), rp=gu.to_np(rp), ci=gu.to_np(ci))


def test_block_rho_all_columns(d64):
    w = d64["w"]
    cols = block.columns(w)
    N = pipeline.scalars(cols, d64["mu"], w.kT, w.n_electrons)["N"]
    assert abs(N - w.n_electrons) < 1e-8                    # the GPU's mu is a valid root
    _, _, rho, rhoE = pipeline.assemble(w, cols, d64["mu"])
    assert np.abs(d64["rho"] - rho).max() < gu.RHO_TOL
    assert np.abs(d64["rhoE"] - rhoE).max() < gu.RHO_TOL


def test_block_energies(d64):
    w = d64["w"]
    sc = pipeline.scalars(block.columns(w), d64["mu"], w.kT, w.n_electrons)
    assert abs(d64["e_band"] - sc["E_band"]) / w.n_atoms < gu.E_TOL_PER_ATOM
    assert abs(d64["f_free"] - sc["F_free"]) / w.n_atoms < gu.E_TOL_PER_ATOM


def test_block_space_of_full_dimension_is_exact(eg):
    w = gu.fragment(16)                                      # nu = M = 64
    s = eg.system_for(w, krylov_block=True)
    ref = pipeline.dense_reference(w)
    s.green_columns()
    rho, rhoE = s.density_matrix(ref["mu"])
    rp, ci = s.pattern()
    rp, ci = gu.to_np(rp), gu.to_np(ci)
    mask = hamiltonian.bsr_to_dense(rp, ci, np.ones((len(ci), 4, 4))) > 0
    assert np.abs(hamiltonian.bsr_to_dense(rp, ci, gu.to_np(rho)) - ref["rho"])[mask].max() < 1e-8
    assert np.abs(hamiltonian.bsr_to_dense(rp, ci, gu.to_np(rhoE)) - ref["rhoE"])[mask].max() < 1e-8


def test_block_diamond4096_sampled_atoms(eg):
    w = dataclasses.replace(wl.make("diamond_4096"), nu=32)
    s = eg.system_for(w, krylov_block=True)
    mu, _, _, _ = s.energy_force()
    rho, rhoE = s.density_matrix(mu)
    rp, ci = s.pattern()
    atoms = [0, 1234, 4095]
    dr, dE = gu.max_rho_diff(gu.to_np(rho), gu.to_np(rhoE), gu.to_np(rp), gu.to_np(ci),
                             _oracle_cols(w, atoms, mu))
    assert dr < gu.RHO_TOL and dE < gu.RHO_TOL


def test_block_breakdown_on_a_dimer(eg):
    """The block space of a dimer atom is the whole 8-dimensional space: the build stops there
    (warning status), and the result is exact."""
    pos, box = wl.dimer(1.5)
    w = wl.Workload("dimer", pos, box, wl.sk_params(), r_cluster=0.0, nu=16)
    s = eg.system_for(w, krylov_block=True)
    assert s.green_columns() == 1                            # ELSES_WARN_BREAKDOWN
    nu_eff = gu.to_np(s.spectra()["nu_eff"])
    assert (nu_eff == 8).all()


def test_exact_gradient_refuses_block_spaces(eg, d64):
    with pytest.raises(eg.ElsesError) as e:
        d64["sys"].omega_gradient(d64["mu"])
    assert e.value.code == -8
