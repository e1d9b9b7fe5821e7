"""The allocation-free bisection entry point (elses_find_mu_static) against elses_find_mu.

Some callers cannot allocate device memory when they need the chemical potential (their own
allocator holds the device memory, or allocation is not allowed in their loop); this entry
point serves them with a static device scratch array. Collected last on purpose, so that a
run stopping at its first failure has already run every other test; it also passes alone.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["diamond_64", "diamond_4096"])
def test_find_mu_static_matches_find_mu_on_two_calls(name):
    eg = gu.library()
    w = wl.make(name)
    s = eg.system_for(w)
    s.green_columns()
    mu_ref, n_ref = s.find_mu()
    e_ref = s.energies(mu_ref)["E_band"]
    mu_tol = gu.mu_tolerance(s, mu_ref)
    sp = s.spectra()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    results = []
    for call, stream in enumerate((None, None, side)):
        free_before = torch.cuda.mem_get_info()[0]
        mu, n, e = eg.find_mu_static(sp["eps"], sp["c"], sp["d"], sp["nu_eff"], w.kT,
                                     w.n_electrons, g=sp["g"], stream=stream)
        if call >= 1:       # after the first call (which may load the device code) nothing moves
            assert torch.cuda.mem_get_info()[0] == free_before
        # two bisections with mu_tol = 1e-13 end within half a bracket of their own crossing
        # of N_e; the crossings differ by the rounding of two summation orders (the static
        # entry sums every pole, the system keeps the poles near mu once the bracket is narrow)
        assert abs(mu - mu_ref) <= mu_tol
        assert abs(n - n_ref) <= 1e-8
        assert abs(e - e_ref) / w.n_atoms <= gu.E_TOL_PER_ATOM
        results.append((mu, n, e))
    # the same kernels in the same order on the same data: equal bit for bit on every call and
    # stream (the shared array is reset where it must start at zero)
    assert results[0] == results[1] == results[2]
    s.close()


def test_find_mu_static_rejects_bad_sizes():
    eg = gu.library()
    t = torch.zeros((4, 8), dtype=torch.float64, device="cuda")
    nu = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(eg.ElsesError) as err:
        eg.find_mu_static(t, t, t, nu, 0.1, 1.0, mu_tol=0.0)      # every pole empty: no bracket
    assert err.value.code in (-3, -4)
    big = torch.zeros((4, 65), dtype=torch.float64, device="cuda")
    with pytest.raises(eg.ElsesError) as err:
        eg.find_mu_static(big, big, big, nu, 0.1, 1.0)
    assert err.value.code == -1
