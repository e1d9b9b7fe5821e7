"""Pins of the oracle's exact gradient through the truncated Krylov build (oracle.adjoint).

Pinned to things other than itself: high-precision divided differences of w, central finite
differences of the independent numpy column path, the full-subspace identity dOmega/dH = rho,
dOmega/dS = -rhoE of exact diagonalisation, and translation invariance of the forces.
"""
import dataclasses

import mpmath
import numpy as np
import pytest

import workloads as wl
from oracle import adjoint, hamiltonian, krylov, physics, pipeline
from oracle.structure import cluster

SK = wl.sk_params()


def _fragment(n_atoms, nu):
    """Isolated piece of displaced diamond in a 30 A box; cluster = whole (M = 4 n_atoms)."""
    pos, _ = wl.diamond((2, 2, 2), sigma=0.05)
    c = pos.mean(axis=0)
    keep = np.sort(np.argsort(np.linalg.norm(pos - c, axis=1))[:n_atoms])
    return wl.Workload(f"fragment_{n_atoms}", pos[keep] - c + 15.0, np.full(3, 30.0), SK,
                       r_cluster=0.0, nu=nu)


def _numpy_omega(Hc, Sc, jl, nu, mu, kT):
    kc = krylov.arnoldi_column(Hc, Sc, jl, nu)
    e, V = krylov.projected_eig(kc.Hp, kc.Sp)
    c, d, _ = krylov.spectra(kc, V, jl)
    return float(np.sum(d * c * physics.omega(e, mu, kT)))


def test_divided_differences_match_high_precision():
    mu, kT = 0.3, 0.1
    rng = np.random.default_rng(11)
    e0 = 0.31
    e = np.concatenate([rng.uniform(-15.0, 10.0, 12), [e0, e0 + 1e-12, e0 + 1e-9, e0 + 1e-6,
                                                        e0 + 1e-3, e0 + 0.05, e0, 4.0, 4.0 + 1e-7]])
    G = adjoint.omega_divided_differences(e, mu, kT)
    mpmath.mp.dps = 60

    def w(x):
        return -2 * kT * mpmath.log(1 + mpmath.exp(-(x - mu) / kT))

    for k in range(len(e)):
        for m in range(len(e)):
            a, b = mpmath.mpf(float(e[k])), mpmath.mpf(float(e[m]))
            ref = 2 / (1 + mpmath.exp((a - mu) / kT)) if a == b else (w(a) - w(b)) / (a - b)
            assert abs(G[k, m] - float(ref)) <= 1e-14 * max(1.0, abs(float(ref))), (k, m)


@pytest.fixture(scope="module")
def frag16():
    w = _fragment(16, nu=10)
    H, S = hamiltonian.dense(w.pos, w.box, w.sk)
    return w, H, S


def test_column_omega_matches_numpy_path(frag16):
    w, H, S = frag16
    mu = 0.4
    for jl in (0, 13, 38, 63):
        om, _, _ = adjoint.column_gradient(H, S, jl, w.nu, mu, w.kT)
        assert abs(om - _numpy_omega(H, S, jl, w.nu, mu, w.kT)) < 1e-12


def test_column_gradient_matches_finite_differences(frag16):
    """Directional derivatives along random symmetric perturbations on the pattern of H, S,
    against fourth-order central differences of the numpy column path (truncated nu = 10)."""
    w, H, S = frag16
    mu, h = 0.4, 1e-4
    rng = np.random.default_rng(5)
    mask = (H != 0) | (S != 0)
    for jl in (1, 22, 50):
        _, gH, gS = adjoint.column_gradient(H, S, jl, w.nu, mu, w.kT)
        for _ in range(2):
            dH = rng.standard_normal(H.shape) * mask
            dS = 0.1 * rng.standard_normal(H.shape) * mask
            dH, dS = dH + dH.T, dS + dS.T

            def om(t):
                return _numpy_omega(H + t * dH, S + t * dS, jl, w.nu, mu, w.kT)

            fd = (8 * (om(h) - om(-h)) - (om(2 * h) - om(-2 * h))) / (12 * h)
            an = float(np.sum(gH * dH) + np.sum(gS * dS))
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (jl, fd, an)


def test_full_subspace_gradient_is_the_density_matrix():
    """With nu = M and the cluster = the whole system, Omega is the exact grand potential and
    dOmega/dH = rho, dOmega/dS = -rhoE of exact diagonalisation."""
    w = _fragment(16, nu=64)
    ref = pipeline.dense_reference(w)
    rp, ci, dH, dS, om = adjoint.pattern_gradient(w, ref["mu"])
    mask = hamiltonian.bsr_to_dense(rp, ci, np.ones_like(dH)) > 0
    assert np.abs(hamiltonian.bsr_to_dense(rp, ci, dH) - ref["rho"])[mask].max() < 1e-8
    assert np.abs(hamiltonian.bsr_to_dense(rp, ci, dS) + ref["rhoE"])[mask].max() < 1e-8
    assert abs(om - ref["Omega"]) / w.n_atoms < 1e-9


@pytest.fixture(scope="module")
def truncated():
    """Periodic 64-atom diamond, 3 A clusters (about 29 atoms), nu = 8: truncated Krylov."""
    pos, box = wl.diamond((2, 2, 2), sigma=0.05)
    w = wl.Workload("diamond_64_rc3", pos, box, SK, r_cluster=3.0, nu=8)
    cols = pipeline.columns(w)
    mu, _ = pipeline.chemical_potential(cols, w.n_electrons, w.kT)
    return w, cols, mu, adjoint.exact_forces(w, mu)


def test_exact_forces_match_finite_differences_at_truncated_nu(truncated):
    w, cols, mu, F = truncated
    h = 1e-4
    checked = 0
    for K, m in ((3, 0), (17, 2), (40, 1), (58, 2)):
        # columns whose cluster holds K: those of the atoms within r_cluster of K
        affected = [4 * J + a for J in cluster(w.pos, w.box, K, w.r_cluster) for a in range(4)]
        members = {}

        def om(t):
            p = w.pos.copy()
            p[K, m] += t
            w2 = dataclasses.replace(w, pos=p)
            members[t] = [tuple(cluster(p, w.box, j // 4, w.r_cluster)) for j in affected[::4]]
            return pipeline.scalars(pipeline.columns(w2, affected), mu, w.kT, w.n_electrons)["Omega"]

        vals = {t: om(t) for t in (h, -h, 2 * h, -2 * h, 0.0)}
        if any(members[t] != members[0.0] for t in members):
            continue      # a cluster boundary is crossed: Omega is not differentiable there
        fd = -(8 * (vals[h] - vals[-h]) - (vals[2 * h] - vals[-2 * h])) / (12 * h)
        assert abs(F[K, m] - fd) <= 1e-6 * np.abs(F).max(), (K, m, F[K, m], fd)
        checked += 1
    assert checked >= 3


def test_exact_forces_differ_from_hellmann_feynman_at_truncated_nu(truncated):
    """The test above has teeth: at nu = 8 the rho-only adjoint is visibly off."""
    w, cols, mu, F = truncated
    rp, ci, rho, rhoE = pipeline.assemble(w, cols, mu)
    F_hf = physics.forces(w.pos, w.box, w.sk, rp, ci, rho, rhoE)
    assert np.abs(F_hf - F).max() > 1e-3 * np.abs(F).max()


def test_exact_forces_sum_to_zero(truncated):
    """Translation invariance: every block depends on R_J - R_I only."""
    _, _, _, F = truncated
    assert np.abs(F.sum(axis=0)).max() < 1e-9 * np.abs(F).max() * len(F)
