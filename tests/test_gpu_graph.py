"""The graph form of elses_energy_force (params.graph): the step captured once as a CUDA graph
and replayed. Its results equal the eager path's bit for bit (the same kernels and arguments,
mu read from device memory instead of the host copy of the same value)."""
import numpy as np
import pytest
import torch

import workloads as wl
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eg():
    return gu.library()


def _same(ra, rb):
    """mu, E_band, F_free and the forces bit for bit (the exact gradient sums its per-column
    contributions as exact fixed-point integers, so its forces do not depend on the order of the
    atomics either)."""
    return (ra[0] == rb[0] and ra[1] == rb[1] and ra[2] == rb[2]
            and np.array_equal(gu.to_np(ra[3]), gu.to_np(rb[3])))


@pytest.mark.parametrize("kw", [{}, {"two_pass": True}, {"exact_forces": True}, {"schedule": 1},
                                {"krylov_block": True}, {"batch_atoms": 16},
                                {"reorth": 1, "schedule": 1}, {"reorth": 1, "exact_forces": True}],
                         ids=["stored", "two_pass", "exact_forces", "batched", "block", "batches",
                              "one_sweep", "one_sweep_exact"])
def test_replay_equals_eager(eg, kw):
    w = wl.make("diamond_64")
    a = eg.system_for(w, **kw)
    ra = a.energy_force()
    rho_a, rhoE_a = a.density_matrix(ra[0])
    b = eg.system_for(w, graph=True, timing=True, **kw)
    for call in range(3):                 # eager, then capture + replay, then replay
        rb = b.energy_force()
        assert _same(ra, rb), call
    st = b.stats()
    assert st["t_krylov_ms"] > 0 and st["bisect_steps"] > 0
    rho_b, rhoE_b = b.density_matrix(rb[0])
    assert np.array_equal(gu.to_np(rho_a), gu.to_np(rho_b))
    assert np.array_equal(gu.to_np(rhoE_a), gu.to_np(rhoE_b))


def test_graph_follows_rebuilds(eg):
    """A rebuild at the same positions keeps the plan (the graph is replayed); moved atoms give
    the eager result at the new positions either way."""
    w = wl.make("diamond_64")
    pos = torch.tensor(w.pos, dtype=torch.float64, device="cuda")
    b = eg.system_for(w, graph=True)
    for _ in range(3):
        b.rebuild(pos)
        rb = b.energy_force()
    a = eg.system_for(w)
    assert _same(a.energy_force(), rb)
    gen = np.random.default_rng(7)
    moved = torch.tensor(w.pos + gen.normal(0.0, 0.02, w.pos.shape), dtype=torch.float64, device="cuda")
    b.rebuild(moved)
    rb = b.energy_force()
    a.rebuild(moved)
    assert _same(a.energy_force(), rb)
    rb = b.energy_force()                 # replayed at the moved positions
    assert _same(a.energy_force(), rb)


def test_calls_after_a_replayed_rebuild_see_its_columns(eg):
    """After a rebuild and a replayed step, the other entry points see that step's columns: the
    density matrix, the spectra and G(z) (which needs V, left to the kept eigen-factors by the
    step) equal those of an eager system at the same positions, bit for bit. The COHP spectrum
    reads the stored columns without recomputing them, so it sees a stale V if the replay left
    the wrong host state."""
    w = wl.make("diamond_64")
    pos = torch.tensor(w.pos, dtype=torch.float64, device="cuda")
    b = eg.system_for(w, graph=True)
    for _ in range(3):                    # eager, capture + replay, replay
        b.rebuild(pos)
        rb = b.energy_force()
    a = eg.system_for(w)
    ra = a.energy_force()
    assert _same(ra, rb)
    for x, y in zip(a.density_matrix(ra[0]), b.density_matrix(rb[0])):
        assert torch.equal(x, y)
    sa, sb = a.spectra(), b.spectra()
    assert all(torch.equal(sa[k], sb[k]) for k in sa)
    zs = [0.3 + 0.2j, -4.0 + 0.1j]
    ca, cb = a.cohp_spectrum(zs), b.cohp_spectrum(zs)
    assert all(torch.equal(x, y) for x, y in zip(ca[:3], cb[:3])) and np.array_equal(ca[3], cb[3])

