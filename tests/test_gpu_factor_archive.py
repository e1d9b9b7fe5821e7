"""Eigen-factors kept across batches (params.keep_factors). With several batches and
keep_factors set, the stored workflow keeps every column's factors -- the Householder
reflectors and L packed, the recorded Givens rotations in a pool shared by all columns --
instead of forming V per batch. The density then replays the same factors with the same
arithmetic as one batch of every atom does, so its results equal that batch's bit for bit, and
so does V where a later call forms it from them. V formed per batch (keep_factors = 0, the
default) agrees to rounding. A pool too small for every column's rotations forms V for the
columns it cannot hold: the spectra, and so mu, are unchanged, and the density agrees to
rounding."""
import numpy as np
import pytest
import torch

import workloads as wl
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

BATCH = 100   # the 512-atom diamond in six batches, the last of 12 atoms


@pytest.fixture(scope="module")
def eg():
    return gu.library()


@pytest.fixture(scope="module")
def ref(eg):
    """One batch of every atom: the factors stay in the batch buffers."""
    w = wl.make("diamond_512")
    s = eg.system_for(w)
    r = s.energy_force()
    rho, rhoE = s.density_matrix(r[0])
    st = s.stats()
    assert st["batches"] == 1 and st["keep_factors"] == 0
    return dict(w=w, s=s, r=r, F=gu.to_np(r[3]), rho=gu.to_np(rho), rhoE=gu.to_np(rhoE))


def _same(ref, r):
    return (r[0] == ref["r"][0] and r[1] == ref["r"][1] and r[2] == ref["r"][2]
            and np.array_equal(gu.to_np(r[3]), ref["F"]))


def _close(ref, s, r, rel=1e-12):
    assert abs(r[0] - ref["r"][0]) <= gu.mu_tolerance(s, r[0])
    assert abs(r[1] - ref["r"][1]) <= rel * abs(ref["r"][1])
    F = gu.to_np(r[3])
    assert np.abs(F - ref["F"]).max() <= 1e-10 * np.abs(ref["F"]).max()
    rho, rhoE = s.density_matrix(ref["r"][0])
    assert np.abs(gu.to_np(rho) - ref["rho"]).max() <= 1e-13 * np.abs(ref["rho"]).max()
    assert np.abs(gu.to_np(rhoE) - ref["rhoE"]).max() <= 1e-13 * np.abs(ref["rhoE"]).max()


def test_kept_factors_equal_one_batch(eg, ref):
    s = eg.system_for(ref["w"], batch_atoms=BATCH, keep_factors=1)
    r = s.energy_force()
    st = s.stats()
    assert st["batches"] == 6 and st["keep_factors"] == 1
    assert st["kept_rotations"] > 0 and st["v_formed_columns"] == 0
    assert _same(ref, r)
    rho, rhoE = s.density_matrix(r[0])
    assert np.array_equal(gu.to_np(rho), ref["rho"]) and np.array_equal(gu.to_np(rhoE), ref["rhoE"])
    r2 = s.energy_force()                 # a second pass starts the pool afresh
    assert _same(ref, r2) and s.stats()["kept_rotations"] == st["kept_rotations"]


def test_v_per_batch_agrees_to_rounding(eg, ref):
    s = eg.system_for(ref["w"], batch_atoms=BATCH)
    r = s.energy_force()
    st = s.stats()
    assert st["batches"] == 6 and st["keep_factors"] == 0 and st["kept_rotations"] == 0
    _close(ref, s, r)


@pytest.mark.parametrize("per_column", [2, 400])
def test_small_pool_forms_v_for_the_rest(eg, ref, per_column):
    """A pool of 2 or 400 rotations per column (a column needs several hundred): V is formed
    for almost every column, or for part of them."""
    s = eg.system_for(ref["w"], batch_atoms=BATCH, keep_factors=per_column)
    r = s.energy_force()
    st = s.stats()
    assert st["keep_factors"] == 1 and st["v_formed_columns"] > 0
    assert st["kept_rotations"] <= per_column * 4 * ref["w"].n_atoms
    if per_column == 400:
        assert st["kept_rotations"] > 0 and st["v_formed_columns"] < 4 * ref["w"].n_atoms
    assert r[0] == ref["r"][0]            # the spectra do not depend on where the factors go
    _close(ref, s, r)


def test_v_formed_from_the_archive(eg, ref):
    """Calls that need V itself (G(z) through the COHP spectrum, the spectra) form it from the
    kept factors with the arithmetic of one batch: bit for bit."""
    s = eg.system_for(ref["w"], batch_atoms=BATCH, keep_factors=1)
    assert _same(ref, s.energy_force())
    zs = [0.3 + 0.2j, -4.0 + 0.1j]
    ca, cb = ref["s"].cohp_spectrum(zs), s.cohp_spectrum(zs)
    assert all(torch.equal(x, y) for x, y in zip(ca[:3], cb[:3])) and np.array_equal(ca[3], cb[3])
    sa, sb = ref["s"].spectra(), s.spectra()
    assert all(torch.equal(sa[k], sb[k]) for k in sa)
    rho, _ = s.density_matrix(ref["r"][0])  # now from V: the same to rounding
    assert np.abs(gu.to_np(rho) - ref["rho"]).max() <= 1e-13 * np.abs(ref["rho"]).max()


def test_exact_forces_from_the_archive(eg, ref):
    """The exact gradient reads V: formed from the kept factors, the forces equal one batch's."""
    a = eg.system_for(ref["w"], exact_forces=True)
    b = eg.system_for(ref["w"], exact_forces=True, batch_atoms=BATCH, keep_factors=1)
    ra, rb = a.energy_force(), b.energy_force()
    assert ra[0] == rb[0] and ra[1] == rb[1]
    assert np.array_equal(gu.to_np(ra[3]), gu.to_np(rb[3]))


def test_graph_replay_with_kept_factors(eg, ref):
    s = eg.system_for(ref["w"], batch_atoms=BATCH, graph=True, keep_factors=1)
    for call in range(3):                 # eager, capture + replay, replay
        assert _same(ref, s.energy_force()), call
    rho, _ = s.density_matrix(ref["r"][0])
    assert np.array_equal(gu.to_np(rho), ref["rho"])


def test_partial_passes_and_g_of_z(eg, ref):
    """Columns recomputed after a full pass take fresh runs of the pool (the others keep
    theirs); a batch recomputed for G(z) forms its V, and its columns leave the archive. On the
    one-batch system the same G(z) range starts inside its batch, which is then recomputed from
    its first atom (a range that did not start a planned batch once skipped the Krylov build)."""
    s = eg.system_for(ref["w"], batch_atoms=BATCH, keep_factors=1)
    assert _same(ref, s.energy_force())
    used = s.stats()["kept_rotations"]
    s.green_columns(4 * 100, 4 * 250)     # two batches, the second ragged
    assert s.stats()["kept_rotations"] > used
    mu, _ = s.find_mu()
    assert mu == ref["r"][0]
    rho, rhoE = s.density_matrix(mu)
    assert np.array_equal(gu.to_np(rho), ref["rho"]) and np.array_equal(gu.to_np(rhoE), ref["rhoE"])
    G = s.green_columns(4 * 300, 4 * 400, z=[0.1 + 0.3j])
    Gr = ref["s"].green_columns(4 * 300, 4 * 400, z=[0.1 + 0.3j])
    assert torch.equal(G, Gr)
    rho, _ = s.density_matrix(mu)
    assert np.abs(gu.to_np(rho) - ref["rho"]).max() <= 1e-13 * np.abs(ref["rho"]).max()



def test_block_spaces_with_kept_factors(eg, ref):
    """Block-start spaces give every column its own projected problem too: kept across six
    batches, the results equal one batch's bit for bit."""
    a = eg.system_for(ref["w"], krylov_block=True)
    b = eg.system_for(ref["w"], krylov_block=True, batch_atoms=BATCH, keep_factors=1)
    ra, rb = a.energy_force(), b.energy_force()
    assert b.stats()["keep_factors"] == 1
    assert ra[0] == rb[0] and ra[1] == rb[1] and ra[2] == rb[2]
    assert np.array_equal(gu.to_np(ra[3]), gu.to_np(rb[3]))
