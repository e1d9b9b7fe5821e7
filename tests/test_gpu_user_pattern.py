"""elses_set_hs on a caller's block pattern (Eq. 1 with caller H and S): the sparse products,
rho and the band energy follow the caller's pattern, against the oracle's column path on the
same dense matrices; malformed patterns are rejected before anything changes."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import hamiltonian, pipeline, structure
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

R_WIDE = 3.2        # the caller's pattern: every pair within 3.2 A (the library's is 2.6 A)


@pytest.fixture(scope="module")
def eg():
    return gu.library()


def _wide_values(w, rp, ci, seed=3):
    """Slater-Koster H, S on the wide pattern plus seeded symmetric couplings on the blocks
    beyond r_cut (where the Slater-Koster integrals vanish): H by up to 0.3 eV, S by up to 0.01."""
    H, S = hamiltonian.bsr_values(w.pos, w.box, w.sk, rp, ci)
    tmap = structure.transpose_map(rp, ci)
    rows = np.repeat(np.arange(w.n_atoms), np.diff(rp))
    d = structure.min_image(w.pos[ci] - w.pos[rows], w.box)
    far = np.sqrt(structure.dist2(d)) > w.sk.r_cut
    rng = np.random.default_rng(seed)
    for e in np.nonzero(far & (rows < ci))[0]:
        bh = rng.uniform(-0.3, 0.3, (4, 4))
        bs = rng.uniform(-0.01, 0.01, (4, 4))
        H[e] += bh
        H[tmap[e]] += bh.T
        S[e] += bs
        S[tmap[e]] += bs.T
    return H, S


def _oracle_rho(w, rp, ci, H, S, cols, mu, r_cluster):
    out = {}
    for j in cols:
        J = int(j) // 4
        atoms = structure.cluster(w.pos, w.box, J, r_cluster)
        Hc = hamiltonian.bsr_submatrix(rp, ci, H, atoms)
        Sc = hamiltonian.bsr_submatrix(rp, ci, S, atoms)
        col = pipeline.solve_column_matrices(Hc, Sc, atoms, ci[rp[J]:rp[J + 1]], j, w.nu)
        r, rE = pipeline.rho_column(col, mu, w.kT)
        out[j] = (col, r, rE)
    return out


def _compare(eg, s, w, rp, ci, oc, mu):
    rho, rhoE = s.density_matrix(mu)
    rho, rhoE = gu.to_np(rho), gu.to_np(rhoE)
    for j, (col, r, rE) in oc.items():
        assert np.abs(gu.rho_of_column(rho, rp, ci, j, col.pattern) - r).max() <= gu.RHO_TOL, j
        assert np.abs(gu.rho_of_column(rhoE, rp, ci, j, col.pattern) - rE).max() <= gu.RHOE_TOL, j


def test_wide_pattern_whole_system_cluster(eg):
    """64-atom diamond, cluster = whole system: every column, rho on the caller's pattern and the
    band energy at the GPU's mu against the oracle on the same dense H and S."""
    w = wl.make("diamond_64")
    rp, ci = structure.neighbor_csr(w.pos, w.box, R_WIDE)
    H, S = _wide_values(w, rp, ci)
    assert np.linalg.eigvalsh(hamiltonian.bsr_to_dense(rp, ci, S)).min() > 0.1
    s = eg.system_for(w)
    nnzb0 = s.nnzb
    s.set_hs(torch.tensor(H, device="cuda"), torch.tensor(S, device="cuda"),
             torch.tensor(rp, device="cuda"), torch.tensor(ci, device="cuda"))
    assert s.nnzb == len(ci) > nnzb0
    grp, gci = (gu.to_np(t) for t in s.pattern())
    assert np.array_equal(grp, rp) and np.array_equal(gci, ci)
    s.green_columns()
    mu, n_mu = s.find_mu()
    oc = _oracle_rho(w, rp, ci, H, S, range(4 * w.n_atoms), mu, 0.0)
    cols = [c for c, _, _ in oc.values()]
    assert abs(pipeline.scalars(cols, mu, w.kT, w.n_electrons)["N"] - w.n_electrons) < 1e-8
    _compare(eg, s, w, rp, ci, oc, mu)
    e = s.energies(mu)
    assert abs(e["E_band"] - pipeline.scalars(cols, mu, w.kT, w.n_electrons)["E_band"]) / w.n_atoms \
        <= gu.E_TOL_PER_ATOM
    with pytest.raises(eg.ElsesError) as err:          # forces need the Slater-Koster H, S
        s.energy_force()
    assert err.value.code == -9
    s.rebuild(torch.tensor(w.pos, device="cuda"))      # a rebuild restores the library's pattern
    assert s.nnzb == nnzb0


def test_wide_pattern_local_clusters(eg):
    """4096-atom diamond with 6 A clusters and the 3.2 A pattern: sampled columns against the
    oracle."""
    w = wl.make("diamond_4096")
    rp, ci = structure.neighbor_csr(w.pos, w.box, R_WIDE)
    H, S = _wide_values(w, rp, ci)
    s = eg.system_for(w)
    s.set_hs(torch.tensor(H, device="cuda"), torch.tensor(S, device="cuda"),
             torch.tensor(rp, device="cuda"), torch.tensor(ci, device="cuda"))
    s.green_columns()
    mu, _ = s.find_mu()
    oc = _oracle_rho(w, rp, ci, H, S, wl.sample_columns(4 * w.n_atoms, 24), mu, w.r_cluster)
    _compare(eg, s, w, rp, ci, oc, mu)


def test_malformed_patterns_are_rejected(eg):
    w = wl.make("diamond_64")
    s = eg.system_for(w)
    mu0, e0, _, _ = s.energy_force()
    rp, ci = structure.neighbor_csr(w.pos, w.box, w.sk.r_cut)

    def attempt(rp_, ci_, code=-1):
        z = torch.zeros((len(ci_), 4, 4), dtype=torch.float64, device="cuda")
        with pytest.raises(eg.ElsesError) as err:
            s.set_hs(z, z, torch.tensor(rp_, device="cuda"), torch.tensor(ci_, device="cuda"))
        assert err.value.code == code

    # a block without its transpose: drop block (1, J) for J > 1 from row 1 only
    J = ci[rp[1] + np.nonzero(ci[rp[1]:rp[2]] > 1)[0][0]]
    keep = np.ones(len(ci), bool)
    keep[rp[1] + np.searchsorted(ci[rp[1]:rp[2]], J)] = False
    rp1 = rp.copy()
    rp1[2:] -= 1
    attempt(rp1, ci[keep])
    # a row without its diagonal block
    keep = np.ones(len(ci), bool)
    keep[rp[5] + np.searchsorted(ci[rp[5]:rp[6]], 5)] = False
    rp2 = rp.copy()
    rp2[6:] -= 1
    attempt(rp2, ci[keep])
    # a row out of order
    ci3 = ci.copy()
    ci3[rp[7]], ci3[rp[7] + 1] = ci3[rp[7] + 1], ci3[rp[7]]
    attempt(rp, ci3)
    # nothing changed: the system still gives its results
    mu, e, _, _ = s.energy_force()
    assert mu == mu0 and e == e0


def test_pattern_beyond_the_clusters_is_rejected(eg):
    """With 3.0 A clusters a 3.2 A pattern joins atoms outside each other's clusters: the
    columns' pattern rows would leave their Krylov spaces, so the call is refused."""
    import dataclasses
    w = dataclasses.replace(wl.make("diamond_4096"), r_cluster=3.0)
    rp, ci = structure.neighbor_csr(w.pos, w.box, R_WIDE)
    s = eg.system_for(w)
    z = torch.zeros((len(ci), 4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(eg.ElsesError) as err:
        s.set_hs(z, z, torch.tensor(rp, device="cuda"), torch.tensor(ci, device="cuda"))
    assert err.value.code == -1
