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
