"""Exact gradient through the truncated Krylov method on the GPU (elses_omega_gradient).

Parity with the oracle's autodiff gradient (oracle.adjoint) to 1e-9 relative; the full-subspace
identity dOmega/dH = rho, dOmega/dS = -rhoE; forces against central finite differences of
Omega at fixed mu at nu = 30 to 1e-5 relative (where the density-matrix forces are far off).
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import adjoint, structure
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-9          # relative to the largest gradient entry


@pytest.fixture(scope="module")
def eg():
    return gu.library()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def d64(eg):
    w = wl.make("diamond_64")
    s = eg.system_for(w)
    mu, _, _, _ = s.energy_force()
    dH, dS = s.omega_gradient(mu)
    rp, ci = s.pattern()
    return dict(w=w, sys=s, mu=mu, dH=gu.to_np(dH), dS=gu.to_np(dS), rp=gu.to_np(rp), ci=gu.to_np(ci))


def test_gradient_matches_oracle_all_columns(d64):
    w = d64["w"]
    rp, ci, dH, dS, _ = adjoint.pattern_gradient(w, d64["mu"])
    assert np.array_equal(rp, d64["rp"]) and np.array_equal(ci, d64["ci"])
    assert _rel(d64["dH"], dH) < GRAD_TOL
    assert _rel(d64["dS"], dS) < GRAD_TOL


def test_gradient_of_an_atom_range(eg, d64):
    """The atoms [lo, hi) alone: the same as the oracle's sum over their columns."""
    w, s = d64["w"], d64["sys"]
    dH, dS = s.omega_gradient(d64["mu"], 10, 13)
    _, _, oH, oS, _ = adjoint.pattern_gradient(w, d64["mu"], cols=np.arange(40, 52))
    assert _rel(gu.to_np(dH), oH) < GRAD_TOL
    assert _rel(gu.to_np(dS), oS) < GRAD_TOL


def test_gradient_two_pass_equals_stored(eg, d64):
    w = d64["w"]
    s2 = eg.system_for(w, two_pass=True)
    s2.energy_force()
    dH, dS = s2.omega_gradient(d64["mu"])
    assert np.abs(gu.to_np(dH) - d64["dH"]).max() < 1e-12 * np.abs(d64["dH"]).max()
    assert np.abs(gu.to_np(dS) - d64["dS"]).max() < 1e-12 * np.abs(d64["dS"]).max()


def test_full_subspace_gradient_is_the_density_matrix(eg):
    """nu = M = 64: the Krylov space is the whole space and cannot move, so the gradient is the
    density-matrix adjoint. The reverse sweep then carries only rounding, divided by the last
    (tiny) beta of the exhausted space, hence the looser bound than the 1e-8 of rho itself."""
    w = gu.fragment(16)
    s = eg.system_for(w)
    mu, _, _, _ = s.energy_force()
    rho, rhoE = s.density_matrix(mu)
    dH, dS = s.omega_gradient(mu)
    assert np.abs(gu.to_np(dH) - gu.to_np(rho)).max() < 1e-7
    assert np.abs(gu.to_np(dS) + gu.to_np(rhoE)).max() < 1e-7


@pytest.fixture(scope="module")
def d4096(eg):
    w = wl.make("diamond_4096")
    s = eg.system_for(w, exact_forces=True)
    mu, _, _, F = s.energy_force()
    return dict(w=w, sys=s, mu=mu, F=gu.to_np(F))


def test_diamond4096_sampled_atoms_match_oracle(d4096):
    w, s, mu = d4096["w"], d4096["sys"], d4096["mu"]
    for J in (0, 2345):
        dH, dS = s.omega_gradient(mu, J, J + 1)
        _, _, oH, oS, _ = adjoint.pattern_gradient(w, mu, cols=np.arange(4 * J, 4 * J + 4))
        assert _rel(gu.to_np(dH), oH) < GRAD_TOL, J
        assert _rel(gu.to_np(dS), oS) < GRAD_TOL, J


@pytest.mark.slow
def test_diamond4096_exact_forces_match_finite_differences(eg, d4096):
    """nu = 30: exact forces against fourth-order central differences of Omega at fixed mu, for
    atoms whose clusters do not change within the displacements; the density-matrix forces miss
    by far more than the gate."""
    w, s, mu, F = d4096["w"], d4096["sys"], d4096["mu"], d4096["F"]
    h = 1e-4
    F_hf = gu.to_np(eg.system_for(w).energy_force()[3])
    scale = np.abs(F).max()
    assert abs(F.sum(axis=0)).max() < 1e-9 * scale * len(F)
    probe = eg.system_for(w)
    ref_cl = [tuple(structure.cluster(w.pos, w.box, J, w.r_cluster)) for J in range(w.n_atoms)]
    checked, hf_gap = 0, 0.0
    for K, m in ((7, 0), (1500, 1), (3001, 2), (4095, 0)):
        vals, frozen = {}, True
        for t in (h, -h, 2 * h, -2 * h):
            p = w.pos.copy()
            p[K, m] += t
            near = structure.cluster(p, w.box, K, w.r_cluster)
            frozen &= all(tuple(structure.cluster(p, w.box, J, w.r_cluster)) == ref_cl[J] for J in near)
            frozen &= tuple(near) == ref_cl[K]
            probe.rebuild(torch.as_tensor(p, dtype=torch.float64).cuda())
            probe.green_columns()
            vals[t] = probe.energies(mu)["Omega"]
        if not frozen:
            continue
        fd = -(8 * (vals[h] - vals[-h]) - (vals[2 * h] - vals[-2 * h])) / (12 * h)
        assert abs(F[K, m] - fd) <= 1e-5 * scale, (K, m, F[K, m], fd)
        hf_gap = max(hf_gap, abs(F_hf[K, m] - fd) / scale)
        checked += 1
    assert checked >= 3
    assert hf_gap > 1e-3


def test_kept_bases_equal_recomputed_bases(eg, d64):
    """With exact forces the Krylov pass keeps every column's bases and the adjoint reads them;
    the gradient is the one of the recomputing path (d64 was built without exact forces)."""
    s = eg.system_for(d64["w"], exact_forces=True)
    mu, _, _, _ = s.energy_force()
    assert mu == d64["mu"]
    dH, dS = s.omega_gradient(mu)
    assert np.abs(gu.to_np(dH) - d64["dH"]).max() <= 1e-12 * np.abs(d64["dH"]).max()
    assert np.abs(gu.to_np(dS) - d64["dS"]).max() <= 1e-12 * np.abs(d64["dS"]).max()


@pytest.mark.slow
def test_composite_sampled_atoms_match_oracle(eg):
    """sp2-sp3 composite with nu by cluster size (20 / 30 / 40): sampled atoms of each class."""
    w = wl.make("composite_32768")
    s = eg.system_for(w, exact_forces=True)
    mu, _, _, _ = s.energy_force()
    cp, cidx, _ = s.clusters()
    sizes = np.diff(gu.to_np(cp))
    picks = [int(np.argmin(sizes)), int(np.argmax(sizes)), int(np.argmin(np.abs(sizes - 150)))]
    for J in picks:
        dH, dS = s.omega_gradient(mu, J, J + 1)
        _, _, oH, oS, _ = adjoint.pattern_gradient(w, mu, cols=np.arange(4 * J, 4 * J + 4))
        assert _rel(gu.to_np(dH), oH) < GRAD_TOL, (J, sizes[J])
        assert _rel(gu.to_np(dS), oS) < GRAD_TOL, (J, sizes[J])
