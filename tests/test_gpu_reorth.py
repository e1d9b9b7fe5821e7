"""The second Gram-Schmidt pass from the projected overlap (elses_params.reorth = 1): the
coefficients SU^T (w - U h) of the second classical pass equal -(S' - I) h in exact arithmetic,
so one sweep of the basis subtracts both passes. The space is the same to rounding, and the
results are formed from H' and S' of the basis itself, so they must meet the same gates against
the oracle (two classical passes) as the default path, and agree with it to rounding."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import hamiltonian, pipeline
from tests import gpu_util as gu
from tests.test_gpu_parity import _class_of_atoms, _columns_covering_classes, _sampled_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eg():
    return gu.library()


def test_rho_all_columns_64(eg):
    """Every column of the 64-atom diamond against the oracle, energies included."""
    w = wl.make("diamond_64")
    s = eg.system_for(w, reorth=1)
    mu, e_band, f_free, F = s.energy_force()
    rho, rhoE = s.density_matrix(mu)
    cols = pipeline.columns(w)
    _, _, rho_o, rhoE_o = pipeline.assemble(w, cols, mu)
    assert np.abs(gu.to_np(rho) - rho_o).max() <= gu.RHO_TOL
    assert np.abs(gu.to_np(rhoE) - rhoE_o).max() <= gu.RHOE_TOL
    sc = pipeline.scalars(cols, mu, w.kT, w.n_electrons)
    assert abs(sc["N"] - w.n_electrons) < 1e-8
    assert abs(e_band - sc["E_band"]) / w.n_atoms <= gu.E_TOL_PER_ATOM
    assert abs(f_free - sc["F_free"]) / w.n_atoms <= gu.E_TOL_PER_ATOM


def test_full_subspace_equals_exact_diagonalisation(eg):
    """A 16-atom fragment with nu = M = 64: the space fills the whole system and the last steps
    cancel almost all of H u_n, the case where the one-sweep form orthogonalises least well."""
    w = gu.fragment(16)
    s = eg.system_for(w, reorth=1)
    s.green_columns()
    ref = pipeline.dense_reference(w)
    rho, rhoE = s.density_matrix(ref["mu"])
    rp, ci = (gu.to_np(t) for t in s.pattern())
    mask = hamiltonian.bsr_to_dense(rp, ci, np.ones((len(ci), 4, 4))) > 0
    assert np.abs(hamiltonian.bsr_to_dense(rp, ci, gu.to_np(rho)) - ref["rho"])[mask].max() < 1e-8
    assert np.abs(hamiltonian.bsr_to_dense(rp, ci, gu.to_np(rhoE)) - ref["rhoE"])[mask].max() < 1e-8
    assert abs(s.energies(ref["mu"])["E_band"] - ref["E_band"]) / w.n_atoms < 1e-9


def test_diamond4096_all_columns(eg):
    """All 16384 columns of the 4096-atom system in the production form (work queue, autotuned
    launch shape, CUDA-graph replay) against the oracle; then the default path to rounding."""
    w = wl.make("diamond_4096")
    s = eg.system_for(w, schedule=1, autotune=True, graph=True, reorth=1)
    s.energy_force()                                   # eager, then captured
    s.energy_force()
    r = _sampled_parity(s, w, np.arange(4 * w.n_atoms))   # replayed
    b = eg.system_for(w, schedule=1)
    mu_b, e_b, _, F_b = b.energy_force()
    assert abs(r["mu"] - mu_b) <= gu.mu_tolerance(b, mu_b)
    rho_a, _ = s.density_matrix(r["mu"])
    rho_b, _ = b.density_matrix(r["mu"])
    assert np.abs(gu.to_np(rho_a) - gu.to_np(rho_b)).max() <= 1e-12
    F_b = gu.to_np(F_b)
    assert np.abs(r["F"] - F_b).max() <= 1e-10 * np.abs(F_b).max()
    st = s.stats()
    assert st["krylov_flops"] > 0


def test_flop_count_is_a_third_less_dense_work(eg):
    """The kernel's own count drops by the second pass's dense products (64-atom diamond: every
    column has the whole system as its cluster and runs nu steps)."""
    w = wl.make("diamond_64")
    f = {}
    for ro in (0, 1):
        s = eg.system_for(w, reorth=ro)
        s.reset_stats()
        s.green_columns()
        f[ro] = s.stats()["krylov_flops"]
    nc, nu = 4 * w.n_atoms, w.nu
    drop = sum(4 * (n + 1) * nc - 2 * (n + 1) ** 2 for n in range(nu - 1)) * 4 * w.n_atoms
    assert f[0] - f[1] == drop


def test_half_warp_columns(eg):
    """3.6 A clusters put atoms in classes that run two columns per warp (k_krylov_half)."""
    w = dataclasses.replace(wl.make("diamond_4096"), r_cluster=3.6)
    s = eg.system_for(w, reorth=1)
    assert any(cap % 32 == 16 for cap in s.autotune_shapes())
    _sampled_parity(s, w, wl.sample_columns(4 * w.n_atoms, 256))


def test_composite_sampled_columns(eg):
    """The sp2-sp3 composite: 2048 seeded columns topped up to 32 per size class, with all three
    Krylov dimensions, against the oracle."""
    w = wl.make("composite_32768")
    s = eg.system_for(w, schedule=1, autotune=True, reorth=1)
    caps, cls = _class_of_atoms(s)
    cols, col_cls = _columns_covering_classes(4 * w.n_atoms, cls, 2048, 32)
    r = _sampled_parity(s, w, cols)
    assert set(np.unique(r["nu_eff"])) == {20, 30, 40}


@pytest.mark.slow
def test_amorphous_1m_sampled_columns(eg):
    """The 10^6-atom system in streamed batches: 2048 seeded columns topped up to 32 per size
    class, against the oracle."""
    w = wl.make("amorphous_1m")
    s = eg.system_for(w, schedule=1, reorth=1)
    caps, cls = _class_of_atoms(s)
    cols, col_cls = _columns_covering_classes(4 * w.n_atoms, cls, 2048, 32)
    r = _sampled_parity(s, w, cols)
    for c in caps:
        assert np.sum(col_cls[r["js"]] == c) >= 32, (c, caps)
    assert abs(r["F"].sum(axis=0)).max() < 1e-6


def test_exact_gradient(eg):
    """The exact gradient differentiates the recursion in exact arithmetic, where the second pass
    vanishes: with the one-sweep form it meets the oracle's autodiff gradient (two classical
    passes) at the same 1e-9 gate on every column of the 64-atom diamond; the exact forces agree
    with the default path's to rounding, and the kept bases with the recomputed ones."""
    from oracle import adjoint
    w = wl.make("diamond_64")
    s = eg.system_for(w, reorth=1)
    mu, _, _, _ = s.energy_force()
    dH, dS = (gu.to_np(t) for t in s.omega_gradient(mu))
    _, _, oH, oS, _ = adjoint.pattern_gradient(w, mu)
    assert np.abs(dH - oH).max() <= 1e-9 * np.abs(oH).max()
    assert np.abs(dS - oS).max() <= 1e-9 * np.abs(oS).max()
    a = eg.system_for(w, exact_forces=True, reorth=1)
    b = eg.system_for(w, exact_forces=True)
    ra, rb = a.energy_force(), b.energy_force()
    assert ra[0] == mu                                  # kept bases: the same columns
    Fa, Fb = gu.to_np(ra[3]), gu.to_np(rb[3])
    assert np.abs(Fa - Fb).max() <= 1e-10 * np.abs(Fb).max()
    kH, kS = (gu.to_np(t) for t in a.omega_gradient(mu))
    assert np.abs(kH - dH).max() <= 1e-12 * np.abs(dH).max()
    assert np.abs(kS - dS).max() <= 1e-12 * np.abs(dS).max()


def test_exact_forces_4096_sampled_atoms(eg):
    """The first 8 of the 32 seeded finite-difference atoms of the 4096-atom system: each atom's
    4 columns against the oracle's autodiff."""
    from oracle import adjoint
    w = wl.make("diamond_4096")
    s = eg.system_for(w, exact_forces=True, schedule=1, reorth=1)
    mu, _, _, F = s.energy_force()
    for J in wl.fd_atoms(w.n_atoms)[:8]:
        J = int(J)
        dH, dS = (gu.to_np(t) for t in s.omega_gradient(mu, J, J + 1))
        _, _, oH, oS, _ = adjoint.pattern_gradient(w, mu, cols=np.arange(4 * J, 4 * J + 4))
        assert np.abs(dH - oH).max() <= 1e-9 * np.abs(oH).max(), J
        assert np.abs(dS - oS).max() <= 1e-9 * np.abs(oS).max(), J
    Fb = gu.to_np(eg.system_for(w, exact_forces=True, schedule=1).energy_force()[3])
    assert np.abs(gu.to_np(F) - Fb).max() <= 1e-10 * np.abs(Fb).max()


def test_dimer_breakdown(eg):
    """A z-dimer with nu = 8: the s and pz columns span 4 dimensions, the px and py columns 2, so
    every column breaks down, in the half-warp form with the two columns of a warp stopping at
    different steps; each space is exact on its invariant subspace (rho against the oracle and
    the exact diagonalisation)."""
    pos, box = wl.dimer(wl.sk_params().r0)
    w = wl.Workload("dimer", pos, box, wl.sk_params(), r_cluster=0.0, nu=8)
    s = eg.system_for(w, reorth=1)
    mu, e_band, _, _ = s.energy_force()
    nu = gu.to_np(s.spectra()["nu_eff"])
    assert list(nu[:4]) == [4, 2, 2, 4] and list(nu[4:]) == [4, 2, 2, 4]
    res = pipeline.run(w, mu=mu)
    rho, rhoE = s.density_matrix(mu)
    assert np.abs(gu.to_np(rho) - res["rho"]).max() < gu.RHO_TOL
    assert np.abs(gu.to_np(rhoE) - res["rhoE"]).max() < gu.RHO_TOL
    ref = pipeline.dense_reference(w)
    rp, ci = (gu.to_np(t) for t in s.pattern())
    assert np.abs(hamiltonian.bsr_to_dense(rp, ci, gu.to_np(rho)) - ref["rho"]).max() < 1e-8


def test_indefinite_overlap_is_not_spd(eg):
    """The off-site overlap scaled by 3 makes S indefinite; the one-sweep form meets w^T S w < 0
    and reports ELSES_ERR_NOT_SPD as the two-pass form does."""
    import torch
    w = wl.make("diamond_64")
    s = eg.system_for(w, reorth=1)
    H, S = s.hs()
    rp, ci = (gu.to_np(t) for t in s.pattern())
    onsite = torch.tensor(np.repeat(np.arange(w.n_atoms), np.diff(rp)) == ci, device="cuda")
    s.set_hs(H, torch.where(onsite[:, None, None], S, 3.0 * S))
    with pytest.raises(eg.ElsesError) as err:
        s.green_columns()
    assert err.value.code == -2
    s.set_hs(H, S)
    assert s.green_columns() == 0


def test_block_spaces_keep_two_passes(eg):
    """Block-start spaces have their own build with two classical passes: the setting leaves
    their results unchanged, bit for bit."""
    w = wl.make("diamond_64")
    a = eg.system_for(w, krylov_block=True)
    b = eg.system_for(w, krylov_block=True, reorth=1)
    ra, rb = a.energy_force(), b.energy_force()
    assert ra[0] == rb[0] and ra[1] == rb[1] and np.array_equal(gu.to_np(ra[3]), gu.to_np(rb[3]))


def test_caller_pattern_dense_blocks(eg):
    """Caller H and S on a wider pattern (every pair within 3.2 A, seeded couplings beyond the
    Slater-Koster cutoff): the dense 4 x 4 block products with the one-sweep form, sampled columns
    of the 4096-atom system against the oracle on the same matrices."""
    import torch
    from oracle import structure
    from tests.test_gpu_user_pattern import R_WIDE, _compare, _oracle_rho, _wide_values
    w = wl.make("diamond_4096")
    rp, ci = structure.neighbor_csr(w.pos, w.box, R_WIDE)
    H, S = _wide_values(w, rp, ci)
    s = eg.system_for(w, reorth=1)
    s.set_hs(torch.tensor(H, device="cuda"), torch.tensor(S, device="cuda"),
             torch.tensor(rp, device="cuda"), torch.tensor(ci, device="cuda"))
    s.green_columns()
    mu, _ = s.find_mu()
    oc = _oracle_rho(w, rp, ci, H, S, wl.sample_columns(4 * w.n_atoms, 24), mu, w.r_cluster)
    _compare(eg, s, w, rp, ci, oc, mu)


def test_bad_setting_is_rejected(eg):
    with pytest.raises(eg.ElsesError) as err:
        eg.system_for(wl.make("diamond_64"), reorth=2)
    assert err.value.code == -1
