"""Energy-resolved COHP (Eq. 4 at z = e + i eta) and density of states on the GPU."""
import numpy as np
import pytest

import workloads as wl
from oracle import cohp, pipeline
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

ZS = [0.5 + 0.3j, -6.0 + 0.05j, 3.0 + 1.0j, 0.85 + 0.02j]


@pytest.fixture(scope="module")
def eg():
    return gu.library()


@pytest.fixture(scope="module")
def d64(eg):
    w = wl.make("diamond_64")
    s = eg.system_for(w)
    s.energy_force()
    C, Cs, Cp, dos = s.cohp_spectrum(ZS)
    return dict(w=w, sys=s, C=gu.to_np(C), Cs=gu.to_np(Cs), Cp=gu.to_np(Cp), dos=dos,
                cols=pipeline.columns(w))


def test_cohp_spectrum_matches_oracle(d64):
    oC, oCs, oCp = cohp.cohp_spectrum(d64["w"], d64["cols"], np.array(ZS))
    scale = np.abs(oC).max()
    assert np.abs(d64["C"] - oC).max() <= 1e-10 * scale
    assert np.abs(d64["Cs"] - oCs).max() <= 1e-10 * scale
    assert np.abs(d64["Cp"] - oCp).max() <= 1e-10 * scale


def test_dos_matches_oracle(d64):
    ref = cohp.dos(d64["cols"], np.array(ZS))
    assert np.abs(d64["dos"] - ref).max() <= 1e-11 * np.abs(ref).max()


def test_total_cohp_is_the_band_energy_spectrum(d64):
    sp = {k: gu.to_np(v) for k, v in d64["sys"].spectra().items()}
    z = np.array(ZS)
    ref = np.zeros(len(z))
    for j in range(len(sp["nu_eff"])):
        n = sp["nu_eff"][j]
        gc = sp["g"][j, :n] * sp["c"][j, :n]
        ref += -np.imag(gc[None, :] / (z[:, None] - sp["eps"][j, None, :n])).sum(axis=1) / np.pi
    assert np.abs(d64["C"].sum(axis=0) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_cohp_two_pass_equals_stored(eg, d64):
    s2 = eg.system_for(d64["w"], two_pass=True)
    s2.energy_force()
    C, _, _, dos = s2.cohp_spectrum(ZS, sigma_pi=False)
    assert np.abs(gu.to_np(C) - d64["C"]).max() <= 1e-12 * np.abs(d64["C"]).max()
    assert np.abs(dos - d64["dos"]).max() <= 1e-12 * np.abs(d64["dos"]).max()


def test_lazy_V_survives_a_partial_recompute(eg, d64):
    """After the energy pass V is left unformed; recomputing a few columns first forms V of the
    others from the kept factors, so the spectra on the pattern are unchanged (the recomputed
    columns take their spectra as Q^T z with V: equal to rounding)."""
    s = eg.system_for(d64["w"])
    s.energy_force()
    assert s.green_columns(0, 8) == 0
    C, _, _, dos = s.cohp_spectrum(ZS, sigma_pi=False)
    assert np.abs(gu.to_np(C) - d64["C"]).max() <= 1e-13 * np.abs(d64["C"]).max()
    assert np.abs(dos - d64["dos"]).max() <= 1e-13 * np.abs(d64["dos"]).max()


def test_spectra_are_reproducible(eg, d64):
    """The DOS and the COHP spectrum are fixed-order reductions: a repeat is bit for bit."""
    C, Cs, Cp, dos = d64["sys"].cohp_spectrum(ZS)
    assert np.array_equal(gu.to_np(C), d64["C"]) and np.array_equal(dos, d64["dos"])
    assert np.array_equal(gu.to_np(Cs), d64["Cs"]) and np.array_equal(gu.to_np(Cp), d64["Cp"])
