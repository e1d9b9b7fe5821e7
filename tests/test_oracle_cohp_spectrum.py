"""Pins of the energy-resolved COHP (Eq. 4 at z = e + i eta) and the density of states."""
import numpy as np
import pytest

import workloads as wl
from oracle import cohp, exact, hamiltonian, pipeline

ZS = np.array([0.5 + 0.3j, -6.0 + 0.05j, 3.0 + 1.0j])


@pytest.fixture(scope="module")
def d64():
    w = wl.make("diamond_64")
    return w, pipeline.columns(w)


def test_total_cohp_is_the_band_energy_spectrum(d64):
    """sum over blocks of C_IJ(z) = -(1/pi) Im sum_j sum_k g_k c_k / (z - e_k): the rows of
    H_C in column j lie on the pattern, so the contraction with H gives (H_C Z)_j = g."""
    w, cols = d64
    C, Cs, Cp = cohp.cohp_spectrum(w, cols, ZS)
    ref = np.zeros(len(ZS))
    for c in cols:
        ref += -np.imag((c.g * c.c)[None, :] / (ZS[:, None] - c.eps[None, :])).sum(axis=1) / np.pi
    assert np.abs(C.sum(axis=0) - ref).max() <= 1e-11 * np.abs(ref).max()
    on = np.abs(Cs).sum(axis=1) + np.abs(Cp).sum(axis=1) == 0
    assert np.abs((Cs + Cp)[~on] - C[~on]).max() < 1e-14 * np.abs(C).max()


def test_full_subspace_cohp_and_dos_equal_the_dense_solve():
    pos, _ = wl.diamond((2, 2, 2), sigma=0.05)
    c0 = pos.mean(axis=0)
    keep = np.sort(np.argsort(np.linalg.norm(pos - c0, axis=1))[:16])
    w = wl.Workload("fragment_16", pos[keep] - c0 + 15.0, np.full(3, 30.0), wl.sk_params(),
                    r_cluster=0.0, nu=64)
    cols = pipeline.columns(w)
    H, S = hamiltonian.dense(w.pos, w.box, w.sk)
    rp, ci, G = cohp.green_pattern(w, cols, ZS)
    C, _, _ = cohp.cohp_spectrum(w, cols, ZS)
    Hb, _ = hamiltonian.bsr_values(w.pos, w.box, w.sk, rp, ci)
    e_ex, _ = exact.generalized_eig(H, S)
    for iz, z in enumerate(ZS):
        Gd = np.linalg.solve(z * S - H, np.eye(len(H)))
        Gb = np.zeros((len(ci), 4, 4), dtype=np.complex128)
        for I in range(w.n_atoms):
            for e in range(rp[I], rp[I + 1]):
                J = ci[e]
                Gb[e] = Gd[4 * I:4 * I + 4, 4 * J:4 * J + 4]
        assert np.abs(G[..., iz] - Gb).max() <= 1e-10 * np.abs(Gb).max()
        Cref = -np.einsum("eab,eab->e", Hb, Gb.imag) / np.pi
        assert np.abs(C[:, iz] - Cref).max() <= 1e-10 * np.abs(Cref).max()
    dref = -np.imag(1.0 / (ZS[:, None] - e_ex[None, :])).sum(axis=1) / np.pi
    assert np.abs(cohp.dos(cols, ZS) - dref).max() <= 1e-10 * np.abs(dref).max()
