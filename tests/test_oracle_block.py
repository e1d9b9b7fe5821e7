"""Pins of the block-start Krylov oracle (oracle.block): the alternative reading of the multiple
Arnoldi method in which the 4 orbitals of an atom start one shared Krylov space."""
import numpy as np

import workloads as wl
from oracle import block, hamiltonian, krylov, pipeline

SK = wl.sk_params()


def _fragment(n_atoms, nu):
    pos, _ = wl.diamond((2, 2, 2), sigma=0.05)
    c = pos.mean(axis=0)
    keep = np.sort(np.argsort(np.linalg.norm(pos - c, axis=1))[:n_atoms])
    return wl.Workload(f"fragment_{n_atoms}", pos[keep] - c + 15.0, np.full(3, 30.0), SK,
                       r_cluster=0.0, nu=nu)


def test_single_start_vector_is_the_per_column_build():
    w = wl.make("diamond_64")
    H, S = hamiltonian.dense(w.pos, w.box, w.sk)
    for jl, nu in ((0, 12), (77, 30), (201, 7)):
        a = krylov.arnoldi_column(H, S, jl, nu)
        b = block.block_arnoldi(H, S, [jl], nu)
        assert a.nu_eff == b.nu_eff
        for x, y in ((a.U, b.U), (a.SU, b.SU), (a.HU, b.HU), (a.Hp, b.Hp), (a.Sp, b.Sp)):
            assert np.array_equal(x, y)


def test_single_start_vector_breakdown_matches():
    pos, box = wl.dimer(1.5)
    H, S = hamiltonian.dense(pos, box, SK)
    a = krylov.arnoldi_column(H, S, 1, 8)          # px of a z-dimer: invariant pair, nu_eff 2
    b = block.block_arnoldi(H, S, [1], 8)
    assert a.nu_eff == b.nu_eff == 2
    assert np.array_equal(a.Hp, b.Hp)


def test_block_basis_is_S_orthonormal_and_spans_each_column_space():
    w = wl.make("diamond_64")
    H, S = hamiltonian.dense(w.pos, w.box, w.sk)
    J, nb = 9, 6
    kc = block.block_arnoldi(H, S, [4 * J + a for a in range(4)], 4 * nb)
    assert kc.nu_eff == 4 * nb
    assert np.abs(kc.U.T @ S @ kc.U - np.eye(4 * nb)).max() < 1e-13
    for a in range(4):
        col = krylov.arnoldi_column(H, S, 4 * J + a, nb)
        resid = col.U - kc.U @ (kc.U.T @ S @ col.U)       # S-orthogonal complement part
        assert np.abs(resid).max() < 1e-10


def test_full_block_space_is_exact_diagonalisation():
    """Block space of dimension M = 64 on the 16-atom fragment: rho equals the dense result."""
    w = _fragment(16, nu=64)
    ref = pipeline.dense_reference(w)
    cols = block.columns(w)
    rp, ci, rho, rhoE = pipeline.assemble(w, cols, ref["mu"])
    mask = hamiltonian.bsr_to_dense(rp, ci, np.ones_like(rho)) > 0
    assert np.abs(hamiltonian.bsr_to_dense(rp, ci, rho) - ref["rho"])[mask].max() < 1e-8
    assert np.abs(hamiltonian.bsr_to_dense(rp, ci, rhoE) - ref["rhoE"])[mask].max() < 1e-8


def test_identity_overlap_gives_block_tridiagonal_projection():
    """S = I: the band build is block Lanczos, so H' is banded with half-bandwidth b = 4."""
    w = wl.make("diamond_64")
    H, _ = hamiltonian.dense(w.pos, w.box, w.sk)
    kc = block.block_arnoldi(H, np.eye(len(H)), [40, 41, 42, 43], 32)
    k, m = np.indices(kc.Hp.shape)
    assert np.abs(kc.Hp[np.abs(k - m) > 4]).max() < 1e-12 * np.abs(kc.Hp).max()
    assert np.abs(kc.Hp[np.abs(k - m) == 4]).min() > 1e-6


def test_block_gauss_quadrature_moments():
    """S = I: sum_k c^(a)_k c^(b)_k e_k^p = (E_J^T H^p E_J)_ab for p <= 2 nu_b - 1 (block Gauss
    quadrature), checked against powers of H applied by brute force."""
    w = wl.make("diamond_64")
    H, _ = hamiltonian.dense(w.pos, w.box, w.sk)
    I = np.eye(len(H))
    jls, nb = [12, 13, 14, 15], 5
    kc = block.block_arnoldi(H, I, jls, 4 * nb)
    e, V = krylov.projected_eig(kc.Hp, kc.Sp)
    C = np.stack([krylov.spectra(kc, V, jl)[0] for jl in jls])       # [alpha][k]
    X = I[:, jls]
    for p in range(2 * nb):
        exact = I[:, jls].T @ X                                         # E^T H^p E
        quad = (C * e[None, :] ** p) @ C.T
        assert np.abs(quad - exact).max() <= 1e-10 * max(1.0, np.abs(exact).max()), p
        X = H @ X


def test_starting_vectors_are_orthonormalised_with_a_general_onsite_overlap():
    """A non-identity on-site S block (as user-supplied S may have) couples the starting
    vectors; the basis must still be S-orthonormal."""
    w = wl.make("diamond_64")
    H, S = hamiltonian.dense(w.pos, w.box, w.sk)
    J = 17
    blk = slice(4 * J, 4 * J + 4)
    rng = np.random.default_rng(3)
    X = 0.05 * rng.standard_normal((4, 4))
    S = S.copy()
    S[blk, blk] += X + X.T
    assert np.linalg.eigvalsh(S).min() > 0
    kc = block.block_arnoldi(H, S, list(range(4 * J, 4 * J + 4)), 16)
    assert np.abs(kc.U.T @ S @ kc.U - np.eye(16)).max() < 1e-13
