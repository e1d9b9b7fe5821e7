"""Parity of the CUDA path (through the C ABI) with the oracle, on seeded synthetic systems.

Gates: |delta rho_ij| <= 1e-10 and |delta E|/atom <= 1e-9 eV against the same-algorithm oracle;
exact diagonalisation at full subspace to 1e-8; finite-difference forces to 1e-5 relative;
bit-exact neighbour, cluster and pattern lists. mu is not unique when it falls in a gap (N(mu)
is flat there), so the GPU's mu is checked for validity (the oracle's N at that mu is N_e) and
rho is compared with the oracle evaluated at the GPU's mu.
"""
import dataclasses

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import exact, hamiltonian, physics, pipeline, structure
from tests import gpu_util as gu
from tests import oracle_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eg():
    return gu.library()


# ----------------------------------------------------------------------------- 64-atom diamond
@pytest.fixture(scope="module")
def d64(eg):
    w = wl.make("diamond_64")
    sysg = eg.system_for(w)
    mu, e_band, f_free, F = sysg.energy_force()
    rho, rhoE = sysg.density_matrix(mu)
    rp, ci = sysg.pattern()
    out = dict(w=w, sys=sysg, mu=mu, e_band=e_band, f_free=f_free, F=gu.to_np(F), rho=gu.to_np(rho),
               rhoE=gu.to_np(rhoE), rp=gu.to_np(rp), ci=gu.to_np(ci), spectra={k: gu.to_np(v) for k, v in sysg.spectra().items()})
    out["oracle_cols"] = pipeline.columns(w)
    return out


def test_pattern_is_bit_exact(d64):
    rp, ci = structure.neighbor_csr(d64["w"].pos, d64["w"].box, d64["w"].sk.r_cut)
    assert np.array_equal(rp, d64["rp"]) and np.array_equal(ci, d64["ci"])


def test_hs_blocks_match(d64):
    H, S = d64["sys"].hs()
    Ho, So = hamiltonian.bsr_values(d64["w"].pos, d64["w"].box, d64["w"].sk, d64["rp"], d64["ci"])
    assert np.abs(gu.to_np(H) - Ho).max() < 1e-13
    assert np.abs(gu.to_np(S) - So).max() < 1e-14


def test_mu_is_a_valid_root(d64):
    w = d64["w"]
    N = pipeline.scalars(d64["oracle_cols"], d64["mu"], w.kT, w.n_electrons)["N"]
    assert abs(N - w.n_electrons) < 1e-8


def test_rho_all_columns(d64):
    w = d64["w"]
    cols = d64["oracle_cols"]
    _, _, rho_o, rhoE_o = pipeline.assemble(w, cols, d64["mu"])
    assert np.abs(d64["rho"] - rho_o).max() <= gu.RHO_TOL
    assert np.abs(d64["rhoE"] - rhoE_o).max() <= gu.RHOE_TOL


def test_energies(d64):
    w = d64["w"]
    sc = pipeline.scalars(d64["oracle_cols"], d64["mu"], w.kT, w.n_electrons)
    assert abs(d64["e_band"] - sc["E_band"]) / w.n_atoms <= gu.E_TOL_PER_ATOM
    assert abs(d64["f_free"] - sc["F_free"]) / w.n_atoms <= gu.E_TOL_PER_ATOM
    e = d64["sys"].energies(d64["mu"])
    assert abs(e["N"] - w.n_electrons) < 1e-8


def test_spectra_invariants(d64):
    sp = d64["spectra"]
    for col in d64["oracle_cols"]:
        j = col.j
        nu = int(sp["nu_eff"][j])
        assert nu == col.nu_eff
        assert gu.significant_poles_match(sp["eps"][j, :nu], sp["c"][j, :nu], col.eps, col.c)
        mg = gu.spectral_moments(sp["eps"][j], sp["c"][j] * sp["d"][j], nu)
        mo = gu.spectral_moments(col.eps, col.c * col.d, nu)
        assert np.abs(mg - mo).max() <= 1e-9 * np.maximum(1.0, np.abs(mo)).max()
        mg = gu.spectral_moments(sp["eps"][j], sp["c"][j] * sp["g"][j], nu)
        mo = gu.spectral_moments(col.eps, col.c * col.g, nu)
        assert np.abs(mg - mo).max() <= 1e-9 * np.maximum(1.0, np.abs(mo)).max()


def test_forces_match_oracle_and_sum_to_zero(d64):
    w = d64["w"]
    _, _, rho_o, rhoE_o = pipeline.assemble(w, d64["oracle_cols"], d64["mu"])
    F_o = physics.forces(w.pos, w.box, w.sk, d64["rp"], d64["ci"], rho_o, rhoE_o)
    assert np.abs(d64["F"] - F_o).max() <= 1e-8 * max(1.0, np.abs(F_o).max())
    assert np.abs(d64["F"].sum(axis=0)).max() < 1e-9


def test_green_function_on_pattern(eg, d64):
    w = d64["w"]
    zs = [0.5 + 0.3j, -6.0 + 0.05j]
    G = gu.to_np(d64["sys"].green_columns(z=zs))
    rp, ci = d64["rp"], d64["ci"]
    for col in d64["oracle_cols"][::37]:
        Z = col.UP @ col.V
        J, alpha = divmod(col.j, 4)
        for iz, z in enumerate(zs):
            g_o = (Z @ (col.c / (z - col.eps))).reshape(-1, 4)
            for p, I in enumerate(col.pattern):
                row = ci[rp[I]:rp[I + 1]]
                e = rp[I] + int(np.searchsorted(row, J))
                assert np.abs(G[e, :, alpha, iz] - g_o[p]).max() <= 1e-10 * max(1.0, np.abs(g_o).max())


def test_deterministic_repeat(eg, d64):
    sysg = d64["sys"]
    mu, e_band, f_free, F = sysg.energy_force()
    assert mu == d64["mu"] and e_band == d64["e_band"] and f_free == d64["f_free"]
    assert np.array_equal(gu.to_np(F), d64["F"])


def test_two_pass_equals_stored(eg, d64):
    """Workflow invariance (the memory-saving workflow does not change the results, Eq. 3)."""
    w = d64["w"]
    s2 = eg.system_for(w, two_pass=True)
    mu, e_band, f_free, F = s2.energy_force()
    rho, rhoE = s2.density_matrix(mu)
    assert mu == d64["mu"] and e_band == d64["e_band"]
    assert np.array_equal(gu.to_np(rho), d64["rho"]) and np.array_equal(gu.to_np(F), d64["F"])


@pytest.mark.parametrize("keep_factors", [1, 0], ids=["kept_factors", "v_per_batch"])
def test_two_pass_equals_stored_in_batches(eg, keep_factors):
    """The same workflow invariance with the columns streamed in batches (the 4096-atom system in
    four batches of 1024 atoms, the form the 10^6-atom system runs in). The stored workflow keeps
    every batch's eigen-factors for the density (keep_factors = 1; or, 0, forms V per batch and
    takes the spectra as Q^T z); the memory-saving one keeps only the spectra in its first
    calculation of G and recomputes each batch for the density. So they agree to rounding, not
    bit for bit: mu within the bound a rounding difference of N allows (gu.mu_tolerance),
    energies and rho to 1e-12 relative."""
    w = wl.make("diamond_4096")
    a = eg.system_for(w, batch_atoms=1024, keep_factors=keep_factors)
    b = eg.system_for(w, batch_atoms=1024, two_pass=True)
    ra, rb = a.energy_force(), b.energy_force()
    assert abs(ra[0] - rb[0]) <= gu.mu_tolerance(a, ra[0])
    assert abs(ra[1] - rb[1]) <= 1e-12 * abs(ra[1]) and abs(ra[2] - rb[2]) <= 1e-12 * abs(ra[2])
    Fa, Fb = gu.to_np(ra[3]), gu.to_np(rb[3])
    assert np.abs(Fa - Fb).max() <= 1e-10 * np.abs(Fa).max()
    for x, y in zip(a.density_matrix(ra[0]), b.density_matrix(ra[0])):
        x, y = gu.to_np(x), gu.to_np(y)
        assert np.abs(x - y).max() <= 1e-12 * np.abs(x).max()


def test_factor_density_equals_formed_V(eg, d64):
    """One batch of every atom leaves V unformed: the spectra come from the rotation replay and
    t = V w from the eigen-factors (rotations, reflectors, L^-T). Several batches that form V
    per batch (keep_factors = 0) take the spectra as Q^T z. The same results to rounding; the
    two N(mu) differ by rounding, so mu agrees within the bound that difference allows where N
    is nearly flat (gu.mu_tolerance), and rho is compared at one mu."""
    s2 = eg.system_for(d64["w"], batch_atoms=16)
    mu, e_band, _, F = s2.energy_force()
    assert abs(mu - d64["mu"]) <= gu.mu_tolerance(s2, mu)
    rho, rhoE = s2.density_matrix(d64["mu"])
    assert abs(s2.energies(d64["mu"])["E_band"] - d64["e_band"]) <= 1e-12 * abs(d64["e_band"])
    scale = np.abs(d64["rho"]).max()
    assert np.abs(gu.to_np(rho) - d64["rho"]).max() <= 1e-13 * scale
    assert np.abs(gu.to_np(rhoE) - d64["rhoE"]).max() <= 1e-13 * np.abs(d64["rhoE"]).max()
    assert np.abs(gu.to_np(F) - d64["F"]).max() <= 1e-12 * np.abs(d64["F"]).max()


def test_batched_schedule_equals_plain(eg, d64):
    s2 = eg.system_for(d64["w"], schedule=1)
    mu, e_band, _, F = s2.energy_force()
    assert mu == d64["mu"] and e_band == d64["e_band"] and np.array_equal(gu.to_np(F), d64["F"])


def test_user_supplied_hs_general_onsite_path(eg, d64):
    """elses_set_hs takes the general path (full on-site blocks in the sparse products); with
    the same H, S it must reproduce the Slater-Koster path to rounding."""
    w = d64["w"]
    s2 = eg.system_for(w)
    H, S = s2.hs()
    s2.set_hs(H, S)
    s2.green_columns()
    rho, _ = s2.density_matrix(d64["mu"])
    assert np.abs(gu.to_np(rho) - d64["rho"]).max() <= gu.RHO_TOL
    e = s2.energies(d64["mu"])
    assert abs(e["E_band"] - d64["e_band"]) / w.n_atoms <= gu.E_TOL_PER_ATOM
    with pytest.raises(eg.ElsesError) as err:
        s2.energy_force()
    assert err.value.code == -9


# ----------------------------------------------------------------------------- full subspace
@pytest.fixture(scope="module")
def full(eg):
    w = gu.fragment(16)                 # M = 64 = nu: the Krylov space is the whole space
    sysg = eg.system_for(w)
    sysg.green_columns()
    ref = pipeline.dense_reference(w)
    return w, sysg, ref


def test_full_subspace_equals_exact_diagonalisation(full):
    w, sysg, ref = full
    rho, rhoE = sysg.density_matrix(ref["mu"])
    rp, ci = sysg.pattern()
    rp, ci = gu.to_np(rp), gu.to_np(ci)
    rho_d = hamiltonian.bsr_to_dense(rp, ci, gu.to_np(rho))
    mask = hamiltonian.bsr_to_dense(rp, ci, np.ones((len(ci), 4, 4))) > 0
    assert np.abs(rho_d - ref["rho"])[mask].max() < 1e-8
    rhoE_d = hamiltonian.bsr_to_dense(rp, ci, gu.to_np(rhoE))
    assert np.abs(rhoE_d - ref["rhoE"])[mask].max() < 1e-8
    e = sysg.energies(ref["mu"])
    assert abs(e["E_band"] - ref["E_band"]) / w.n_atoms < 1e-9


def test_full_subspace_green_function_equals_dense_solve(full):
    w, sysg, ref = full
    zs = [0.3 + 0.5j, -7.0 + 0.05j]
    G = gu.to_np(sysg.green_columns(z=zs))
    rp, ci = (gu.to_np(t) for t in sysg.pattern())
    for j in (0, 13, 42, 63):
        J, alpha = divmod(j, 4)
        for iz, z in enumerate(zs):
            g_ref = exact.green_column(ref["H"], ref["S"], z, j)
            for I in range(w.n_atoms):
                row = ci[rp[I]:rp[I + 1]]
                k = np.searchsorted(row, J)
                if k < len(row) and row[k] == J:
                    e = rp[I] + k
                    assert np.abs(G[e, :, alpha, iz] - g_ref[4 * I:4 * I + 4]).max() <= 1e-10 * np.abs(g_ref).max()


def test_full_subspace_forces_match_finite_differences(eg, full):
    """HF forces are the exact gradient at full subspace: compare with central differences of
    Omega at fixed mu (h = 1e-4 A), each side evaluated by the GPU path."""
    w = full[0]
    s = eg.system_for(w)
    mu, _, _, F = s.energy_force()
    F = gu.to_np(F)
    h = 1e-4
    scale = max(1.0, np.abs(F).max())
    for (K, m) in ((0, 0), (5, 1), (11, 2)):
        om = []
        for sgn in (1, -1):
            pos = w.pos.copy()
            pos[K, m] += sgn * h
            t = eg.System(torch.tensor(pos, device="cuda"), w.box, w.sk, w.r_cluster, w.nu, w.kT,
                          w.n_electrons)
            t.green_columns()
            om.append(t.energies(mu)["Omega"])
            t.close()
        fd = -(om[0] - om[1]) / (2 * h)
        assert abs(fd - F[K, m]) <= 1e-5 * scale
    assert np.abs(F.sum(axis=0)).max() < 1e-9


# ----------------------------------------------------------------------------- larger systems
def _sampled_parity(sysg, w, cols):
    """The GPU's rho, rhoE, spectra and per-column band energy against the oracle on the columns
    `cols`, at the GPU's mu (the oracle on every host core; only the sampled blocks and spectra
    rows leave the device)."""
    mu, e_band, f_free, F = sysg.energy_force()
    rho, rhoE = sysg.density_matrix(mu)
    rp, ci = (gu.to_np(t) for t in sysg.pattern())
    oc = oracle_pool.rho_columns(w, cols, mu)
    js = np.array(sorted(oc))
    ids = [oracle_pool.block_ids(rp, ci, j, oc[j][0]) for j in js]
    e_all = torch.as_tensor(np.concatenate(ids), device="cuda")
    a_all = torch.as_tensor(np.concatenate([np.full(len(i), j % 4) for j, i in zip(js, ids)]), device="cuda")
    g_rho = gu.to_np(rho[e_all, :, a_all])
    g_rhoE = gu.to_np(rhoE[e_all, :, a_all])
    o_rho = np.concatenate([oc[j][1] for j in js])
    o_rhoE = np.concatenate([oc[j][2] for j in js])
    dr = float(np.abs(g_rho - o_rho).max())
    dE = float(np.abs(g_rhoE - o_rhoE).max())
    assert dr <= gu.RHO_TOL and dE <= gu.RHOE_TOL, (dr, dE)
    jt = torch.as_tensor(js, device="cuda")
    sp = {k: gu.to_np(v[jt]) for k, v in sysg.spectra().items()}
    f2 = lambda e: 2.0 * physics.fermi(e, mu, w.kT)
    for q, j in enumerate(js):
        _, _, _, nu, eps, c, g, _ = oc[j]
        assert int(sp["nu_eff"][q]) == nu, j
        assert gu.significant_poles_match(sp["eps"][q, :nu], sp["c"][q, :nu], eps, c), j
        # the column's band energy at the GPU's mu
        Eg = np.sum(f2(sp["eps"][q, :nu]) * sp["g"][q, :nu] * sp["c"][q, :nu])
        assert abs(Eg - np.sum(f2(eps) * g * c)) <= gu.E_TOL_PER_ATOM, j
    return dict(sys=sysg, mu=mu, dr=dr, dE=dE, F=gu.to_np(F), rp=rp, ci=ci, oc=oc,
                nu_eff=sp["nu_eff"], js=js)


def _class_of_atoms(sysg):
    """The Krylov size class (cluster capacity in atoms) of every atom."""
    cp, _, _ = sysg.clusters()
    sizes = np.diff(gu.to_np(cp))
    caps = np.array(sorted(sysg.autotune_shapes()))
    return caps, caps[np.searchsorted(caps, sizes)]


def _columns_covering_classes(M, cls, n, per_class, seed=11):
    """The seeded sample of n columns, topped up so that every size class holds per_class."""
    cols = set(int(j) for j in wl.sample_columns(M, n))
    rng = np.random.default_rng(seed)
    col_cls = np.repeat(cls, 4)
    for c in np.unique(cls):
        have = sum(1 for j in cols if col_cls[j] == c)
        pool = np.setdiff1d(np.nonzero(col_cls == c)[0], np.fromiter(cols, int))
        if have < per_class and len(pool):
            cols.update(int(j) for j in rng.choice(pool, size=min(per_class - have, len(pool)), replace=False))
    return np.array(sorted(cols)), col_cls


def test_diamond4096_all_columns(eg):
    """Every one of the 16384 columns of the 4096-atom system (the bench workload)."""
    w = wl.make("diamond_4096")
    sysg = eg.system_for(w)
    r = _sampled_parity(sysg, w, np.arange(4 * w.n_atoms))
    rp, ci = structure.neighbor_csr(w.pos, w.box, w.sk.r_cut)
    assert np.array_equal(rp, r["rp"]) and np.array_equal(ci, r["ci"])
    cp, cidx, mx = sysg.clusters()
    cp, cidx = gu.to_np(cp), gu.to_np(cidx)
    for J in wl.sample_columns(w.n_atoms, 64):
        assert np.array_equal(cidx[cp[J]:cp[J + 1]], structure.cluster(w.pos, w.box, J, w.r_cluster))
    for j in r["js"][::97]:                   # the oracle's clusters are the library's
        assert r["oc"][j][7] == cp[j // 4 + 1] - cp[j // 4]
    assert abs(r["F"].sum(axis=0)).max() < 1e-8


def test_half_warp_columns(eg):
    """Clusters of 3.6 A (about 30 to 45 atoms): the size classes with an odd number of 16-atom
    slots run two columns per warp, one per half-warp (k_krylov_half). They match the oracle on
    sampled columns, and the one-warp-per-column kernel (k3_lanes = 32) to rounding."""
    w = dataclasses.replace(wl.make("diamond_4096"), r_cluster=3.6)
    r = _sampled_parity(eg.system_for(w), w, wl.sample_columns(4 * w.n_atoms, 48))
    caps = r["sys"].autotune_shapes()
    assert any(cap % 32 == 16 for cap in caps), caps          # a half-warp class is in use
    b = eg.system_for(w, k3_lanes=32)
    assert all(cap % 32 == 0 for cap in b.autotune_shapes())
    mu, e_band, _, F = b.energy_force()
    assert abs(mu - r["mu"]) <= gu.mu_tolerance(b, mu)
    rho_a, _ = r["sys"].density_matrix(r["mu"])
    rho_b, _ = b.density_matrix(r["mu"])
    ra, rb = gu.to_np(rho_a), gu.to_np(rho_b)
    assert np.abs(ra - rb).max() <= 1e-12 * np.abs(rb).max()
    assert np.abs(r["F"] - gu.to_np(F)).max() <= 1e-10 * np.abs(gu.to_np(F)).max()


def test_diamond4096_batched_equals_plain(eg):
    w = wl.make("diamond_4096")
    a = eg.system_for(w, schedule=0)
    b = eg.system_for(w, schedule=1)
    ra, rb = a.energy_force(), b.energy_force()
    assert ra[0] == rb[0] and ra[1] == rb[1] and np.array_equal(gu.to_np(ra[3]), gu.to_np(rb[3]))


def test_composite_sampled_columns(eg):
    """The sp2-sp3 composite in the production form (work queue, autotuned launch shape): a
    seeded sample of 2048 columns, topped up so that every Krylov size class in use holds at
    least 32 of them, and all three Krylov dimensions (20 / 30 / 40 by cluster size) occur."""
    w = wl.make("composite_32768")
    sysg = eg.system_for(w, schedule=1, autotune=True)
    caps, cls = _class_of_atoms(sysg)
    cols, col_cls = _columns_covering_classes(4 * w.n_atoms, cls, 2048, 32)
    r = _sampled_parity(sysg, w, cols)
    for c in caps:
        assert np.sum(col_cls[r["js"]] == c) >= 32, (c, caps)
    assert set(np.unique(r["nu_eff"])) == {20, 30, 40}
    nu_all = gu.to_np(sysg.spectra()["nu_eff"])
    assert set(np.unique(nu_all)) == {20, 30, 40}


@pytest.mark.slow
def test_amorphous_1m_sampled_columns(eg):
    """The 10^6-atom system in streamed batches: a seeded sample of 2048 of its 4,194,304
    columns, topped up to 32 per Krylov size class."""
    w = wl.make("amorphous_1m")
    sysg = eg.system_for(w, schedule=1)
    caps, cls = _class_of_atoms(sysg)
    cols, col_cls = _columns_covering_classes(4 * w.n_atoms, cls, 2048, 32)
    r = _sampled_parity(sysg, w, cols)
    for c in caps:
        assert np.sum(col_cls[r["js"]] == c) >= 32, (c, caps)
    assert abs(r["F"].sum(axis=0)).max() < 1e-6


# ----------------------------------------------------------------------------- edge cases
def test_dimer_breakdown_warning(eg):
    pos, box = wl.dimer(wl.sk_params().r0)
    s = eg.System(torch.tensor(pos, device="cuda"), box, wl.sk_params(), 0.0, 8, 0.1, 8.0)
    assert s.green_columns() == eg.WARN_BREAKDOWN
    nu = gu.to_np(s.spectra()["nu_eff"])
    assert nu[1] == 2 and nu[2] == 2                       # px, py: invariant pi pairs


def test_dimer_columns_stop_at_different_steps(eg):
    """A z-dimer with nu = 8: the s and pz columns span 4 dimensions, the px and py columns 2
    (invariant pi pairs). The two columns that share a warp in the half-warp form (s with px, py
    with pz) stop at different Krylov steps; each Krylov space is then exact on its invariant
    subspace, so rho matches the oracle and the exact diagonalisation."""
    pos, box = wl.dimer(wl.sk_params().r0)
    w = wl.Workload("dimer", pos, box, wl.sk_params(), r_cluster=0.0, nu=8)
    s = eg.system_for(w)
    assert any(cap % 32 == 16 for cap in s.autotune_shapes())      # the half-warp form
    mu, e_band, _, _ = s.energy_force()
    nu = gu.to_np(s.spectra()["nu_eff"])
    assert list(nu[:4]) == [4, 2, 2, 4] and list(nu[4:]) == [4, 2, 2, 4]
    res = pipeline.run(w, mu=mu)
    rho, rhoE = s.density_matrix(mu)
    assert np.abs(gu.to_np(rho) - res["rho"]).max() < gu.RHO_TOL
    assert np.abs(gu.to_np(rhoE) - res["rhoE"]).max() < gu.RHO_TOL
    assert abs(e_band - res["E_band"]) / w.n_atoms < gu.E_TOL_PER_ATOM
    ref = pipeline.dense_reference(w)
    rp, ci = (gu.to_np(t) for t in s.pattern())
    dense = hamiltonian.bsr_to_dense(rp, ci, gu.to_np(rho))
    assert np.abs(dense - ref["rho"]).max() < 1e-8 and abs(mu - ref["mu"]) < 1e-8


def test_errors_are_reported(eg):
    w = wl.make("diamond_64")
    pos = torch.tensor(w.pos, device="cuda")
    with pytest.raises(eg.ElsesError) as e:
        eg.System(pos, [4.0, 4.0, 4.0], w.sk, 0.0, 30, 0.1, w.n_electrons)
    assert e.value.code == -1
    with pytest.raises(eg.ElsesError) as e:
        eg.System(pos, w.box, w.sk, 0.0, 65, 0.1, w.n_electrons)
    assert e.value.code == -1
    bad = pos.clone()
    bad[3, 1] = float("nan")
    with pytest.raises(eg.ElsesError) as e:
        eg.System(bad, w.box, w.sk, 0.0, 30, 0.1, w.n_electrons)
    assert e.value.code == -3
    with pytest.raises(eg.ElsesError) as e:
        eg.System(pos, w.box, w.sk, 0.0, 30, 0.1, w.n_electrons, max_neighbors=4)
    assert e.value.code == -10
    s = eg.System(pos, w.box, w.sk, 0.0, 30, 0.1, 10.0 * w.n_electrons)
    with pytest.raises(eg.ElsesError) as e:
        s.energy_force()
    assert e.value.code == -4
    s2 = eg.System(pos, w.box, w.sk, 0.0, 30, 0.1, w.n_electrons)
    with pytest.raises(eg.ElsesError) as e:
        s2.find_mu()
    assert e.value.code == -9


def test_icohp_matches_oracle_and_sums_to_band_energy(eg, d64):
    """(pi)COHP on the GPU (Eqs. 4-8) against the oracle on the same rho; sum B = E_band (Eq. 6)."""
    from oracle import cohp
    w = d64["w"]
    rho = torch.tensor(d64["rho"], device="cuda")
    B, Bs, Bp = (gu.to_np(t) for t in d64["sys"].icohp(rho))
    Bo, Bso, Bpo = cohp.icohp(w.pos, w.box, w.sk, d64["rp"], d64["ci"], d64["rho"])
    assert np.abs(B - Bo).max() < 1e-12 and np.abs(Bs - Bso).max() < 1e-12 and np.abs(Bp - Bpo).max() < 1e-12
    assert abs(B.sum() - d64["e_band"]) / w.n_atoms < 1e-9


def test_autograd_free_energy_backward_is_minus_forces(eg, full):
    """torch.autograd.Function over the library: dF_free/dR from the adjoint kernels equals
    -forces of elses_energy_force, and matches central differences at full subspace."""
    w = full[0]
    s = eg.system_for(w)
    pos = torch.tensor(w.pos, device="cuda", requires_grad=True)
    f_free, e_band = eg.free_energy(pos, s)
    f_free.backward()
    _, e2, f2, F = s.energy_force()
    assert f_free.item() == f2 and e_band.item() == e2
    assert torch.equal(pos.grad, -F)
    h = 1e-4
    for (K, m) in ((1, 2), (9, 0)):
        vals = []
        for sgn in (1, -1):
            p = torch.tensor(w.pos, device="cuda")
            p[K, m] += sgn * h
            vals.append(eg.free_energy(p, s)[0].item())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - pos.grad[K, m].item()) <= 1e-5 * max(1.0, F.abs().max().item())
