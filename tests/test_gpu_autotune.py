"""The autotuner of the Krylov launch shape (elses_autotune): it picks, per cluster size class,
the resident CTAs per SM by timing, and the results do not depend on the shape."""
import numpy as np
import pytest

import workloads as wl
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eg():
    return gu.library()


def _half_classes(shapes):
    """Capacities of the classes whose columns run on half-warps (an odd number of 16-atom slots)."""
    return {cap for cap in shapes if cap % 32 == 16}


@pytest.mark.parametrize("name, r_cluster", [("diamond_4096", None), ("diamond_4096", 4.2)])
def test_autotuned_shape_keeps_results(eg, name, r_cluster):
    """The CTA count and the queue order leave every result the same bit for bit. Moving an odd
    class between half-warp and whole-warp columns changes its reduction trees, so the results
    then agree to rounding. (4.2 A clusters, 60-75 atoms, put atoms in odd classes.)"""
    import dataclasses
    w = wl.make(name)
    if r_cluster:
        w = dataclasses.replace(w, r_cluster=r_cluster)
    s = eg.system_for(w, schedule=1)
    before = s.autotune_shapes()
    mu, e_band, _, F = s.energy_force()
    F = gu.to_np(F)
    shapes = s.autotune()
    assert len(shapes) >= 1
    for atoms, (bps, order) in shapes.items():
        assert atoms % 16 == 0 and 16 <= atoms <= 512 and 1 <= bps <= 16 and order in ("size", "atom")
    assert s.stats()["k3_ctas_per_sm"] in [b for b, _ in shapes.values()]
    assert s.autotune_shapes() == shapes
    mu2, e_band2, _, F2 = s.energy_force()               # columns recomputed with the new shape
    if _half_classes(shapes) == _half_classes(before):
        assert mu2 == mu and e_band2 == e_band and np.array_equal(gu.to_np(F2), F)
    else:
        assert abs(mu2 - mu) <= gu.mu_tolerance(s, mu2) and abs(e_band2 - e_band) <= 1e-12 * abs(e_band)
        assert np.abs(gu.to_np(F2) - F).max() <= 1e-10 * np.abs(F).max()


def test_autotune_at_build(eg):
    w = wl.make("diamond_64")
    a = eg.system_for(w)
    b = eg.system_for(w, autotune=True)
    ra, rb = a.energy_force(), b.energy_force()
    assert ra[0] == rb[0] and ra[1] == rb[1] and np.array_equal(gu.to_np(ra[3]), gu.to_np(rb[3]))


def test_autotune_refused_when_the_shape_is_fixed(eg):
    s = eg.system_for(wl.make("diamond_64"), k3_ctas_per_sm=2)
    with pytest.raises(eg.ElsesError) as err:
        s.autotune()
    assert err.value.code == -9
