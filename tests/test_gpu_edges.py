"""Edge cases through the C ABI: empty and ragged inputs, a single isolated atom (every column an
invariant one-dimensional space), and the argument checks of the newer entry points."""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import pipeline
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eg():
    return gu.library()


def test_empty_system_is_rejected(eg):
    with pytest.raises(eg.ElsesError) as e:
        eg.System(torch.zeros((0, 3), dtype=torch.float64, device="cuda"), [20.0] * 3, wl.sk_params(),
                  0.0, 8, 0.1, 0.0)
    assert e.value.code == -1


def test_single_isolated_atom(eg):
    """One atom in a large box: H e_j = E e_j, so every column stops at nu_eff = 1 with the
    on-site energy as its pole; with 4 electrons 2 f(Es - mu) + 6 f(Ep - mu) = 4 fixes mu."""
    sk = wl.sk_params()
    pos = np.array([[10.0, 10.0, 10.0]])
    w = wl.Workload("atom", pos, np.full(3, 20.0), sk, r_cluster=0.0, nu=8)
    s = eg.system_for(w)
    assert s.green_columns() == eg.WARN_BREAKDOWN
    sp = {k: gu.to_np(v) for k, v in s.spectra().items()}
    assert (sp["nu_eff"] == 1).all()
    assert np.allclose(sp["eps"][:, 0], [sk.Es, sk.Ep, sk.Ep, sk.Ep], atol=1e-14)
    mu, _ = s.find_mu()
    f = lambda e: 1.0 / (1.0 + np.exp((e - mu) / w.kT))
    assert abs(2 * f(sk.Es) + 6 * f(sk.Ep) - 4.0) < 1e-10
    res = pipeline.run(w, mu=mu)
    rho, _ = s.density_matrix(mu)
    assert np.abs(gu.to_np(rho) - res["rho"]).max() < gu.RHO_TOL
    _, e_band, f_free, F = s.energy_force()
    assert abs(e_band - res["E_band"]) < gu.E_TOL_PER_ATOM
    assert np.abs(gu.to_np(F)).max() == 0.0                # no neighbours, no force


def test_ragged_column_ranges_are_rejected(eg):
    s = eg.system_for(wl.make("diamond_64"))
    for b, e in ((1, 8), (0, 6), (8, 4), (0, 260)):
        with pytest.raises(eg.ElsesError) as err:
            s.green_columns(b, e)
        assert err.value.code == -1
    assert s.green_columns(0, 8) == 0                    # whole atoms are fine
    with pytest.raises(eg.ElsesError) as err:            # but mu needs every column
        s.find_mu()
    assert err.value.code == -9


def test_gradient_and_spectrum_arguments(eg):
    s = eg.system_for(wl.make("diamond_64"))
    mu, _, _, _ = s.energy_force()
    for lo, hi in ((-1, 4), (5, 3), (0, 65)):
        with pytest.raises(eg.ElsesError) as err:
            s.omega_gradient(mu, lo, hi)
        assert err.value.code == -1
    with pytest.raises(eg.ElsesError) as err:
        s.cohp_spectrum([])
    assert err.value.code == -1
    dH, dS = s.omega_gradient(mu, 7, 7)                   # an empty atom range is a zero gradient
    assert float(dH.abs().max()) == 0.0 and float(dS.abs().max()) == 0.0


def test_block_space_arguments(eg):
    w = wl.make("diamond_64")
    pos = torch.tensor(w.pos, device="cuda")
    with pytest.raises(eg.ElsesError) as err:
        eg.System(pos, w.box, w.sk, 0.0, 3, 0.1, w.n_electrons, krylov_block=True)
    assert err.value.code == -1
    with pytest.raises(eg.ElsesError) as err:
        eg.System(pos, w.box, w.sk, 0.0, 16, 0.1, w.n_electrons, krylov_block=True, exact_forces=True)
    assert err.value.code == -8


def test_indefinite_overlap_is_not_spd(eg):
    """Eq. 1 needs S positive definite. User values with the off-site overlap scaled by 3 make S
    indefinite (lambda_min < 0, library eigvalsh): the Krylov build meets w^T S w < 0 and
    elses_green_columns reports ELSES_ERR_NOT_SPD instead of a silently truncated space; the
    oracle raises on the same input."""
    from oracle import hamiltonian, krylov
    w = wl.make("diamond_64")
    s = eg.system_for(w)
    H, S = s.hs()
    rp, ci = (gu.to_np(t) for t in s.pattern())
    onsite = torch.tensor(np.repeat(np.arange(w.n_atoms), np.diff(rp)) == ci, device="cuda")
    eye = torch.eye(4, dtype=torch.float64, device="cuda")
    S3 = torch.where(onsite[:, None, None], S, 3.0 * S)
    S3_dense = hamiltonian.bsr_to_dense(rp, ci, gu.to_np(S3))
    assert np.linalg.eigvalsh(S3_dense).min() < -0.1
    assert torch.equal(S[onsite], eye.expand(int(onsite.sum()), 4, 4))
    with pytest.raises(krylov.NotPositiveDefinite):
        krylov.arnoldi_column(hamiltonian.bsr_to_dense(rp, ci, gu.to_np(H)), S3_dense, 0, w.nu)
    s.set_hs(H, S3)
    with pytest.raises(eg.ElsesError) as err:
        s.green_columns()
    assert err.value.code == -2
    s.set_hs(H, S)                                        # the valid overlap builds again
    assert s.green_columns() == 0


def test_column_without_a_space_under_a_sweep_cap(eg):
    """A non-positive diagonal overlap S_jj leaves column j without a Krylov space (nu_eff = 0,
    ELSES_ERR_ARG); with a QR sweep cap set the eigensolver still has nothing to chase for it
    (the cap no longer lets an empty column into the sweep loop), the call reports the error and
    the valid overlap builds again."""
    w = wl.make("diamond_64")
    s = eg.system_for(w, max_qr_sweeps=200)             # enough for every nu = 30 column
    H, S = s.hs()
    rp, ci = (gu.to_np(t) for t in s.pattern())
    e33 = int(np.flatnonzero((np.repeat(np.arange(w.n_atoms), np.diff(rp)) == 3) & (ci == 3))[0])
    Sb = S.clone()
    Sb[e33, 0, 0] = -1.0
    s.set_hs(H, Sb)
    with pytest.raises(eg.ElsesError) as err:
        s.green_columns()
    assert err.value.code in (-1, -2)
    assert int(s.spectra()["nu_eff"][12]) == 0          # column 4 * 3 + 0: no space
    s.set_hs(H, S)
    assert s.green_columns() == 0


def test_qr_sweep_cap_reports_timeout(eg):
    """The implicit-shift QR chase of the projected eigenproblem is a bounded loop: with its cap
    at one sweep per column (a 30 x 30 tridiagonal needs about two per eigenvalue) the columns
    run out and elses_green_columns returns ELSES_ERR_TIMEOUT; nothing waits or spins. With the
    default cap (30 nu) the same system solves."""
    w = wl.make("diamond_64")
    s = eg.system_for(w, max_qr_sweeps=1)
    with pytest.raises(eg.ElsesError) as err:
        s.green_columns()
    assert err.value.code == -5
    s.close()
    assert eg.system_for(w).green_columns() == 0


def test_cluster_capacity(eg):
    """max_cluster bounds the cluster lists: a system whose largest cluster has exactly that many
    atoms runs (results equal the default capacity's bit for bit), one atom fewer is
    ELSES_ERR_CAPACITY at build time, before any column is solved."""
    w = wl.make("diamond_512")
    a = eg.system_for(w)
    cp, _, mx = a.clusters()
    largest = int(np.diff(gu.to_np(cp)).max())
    assert largest == mx
    ra = a.energy_force()
    b = eg.system_for(w, max_cluster=largest)
    rb = b.energy_force()
    assert ra[0] == rb[0] and ra[1] == rb[1] and np.array_equal(gu.to_np(ra[3]), gu.to_np(rb[3]))
    with pytest.raises(eg.ElsesError) as err:
        eg.system_for(w, max_cluster=largest - 1)
    assert err.value.code == -10


@pytest.mark.parametrize("nu", [1, 2, 3])
def test_smallest_krylov_dimensions(eg, nu):
    """nu = 1, 2, 3 (no Householder step, no QR sweep or a single 2 x 2 one): every column of the
    64-atom diamond against the oracle, at the GPU's mu."""
    import dataclasses
    w = dataclasses.replace(wl.make("diamond_64"), nu=nu)
    s = eg.system_for(w)
    mu, e_band, _, _ = s.energy_force()
    cols = pipeline.columns(w)
    assert abs(pipeline.scalars(cols, mu, w.kT, w.n_electrons)["N"] - w.n_electrons) < 1e-8
    rho, rhoE = s.density_matrix(mu)
    _, _, rho_o, rhoE_o = pipeline.assemble(w, cols, mu)
    assert np.abs(gu.to_np(rho) - rho_o).max() <= gu.RHO_TOL
    assert np.abs(gu.to_np(rhoE) - rhoE_o).max() <= gu.RHOE_TOL
    assert np.array_equal(gu.to_np(s.spectra()["nu_eff"]), np.full(4 * w.n_atoms, nu))
