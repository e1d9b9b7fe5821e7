"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *draws inputs*: atomic positions in orthorhombic periodic boxes and the
numbers of a two-centre s/p Slater-Koster parameter set. It holds none of the method's
arithmetic (no Hamiltonian or overlap matrix elements, no Krylov step, no Fermi function),
so that the oracle and the CUDA path can both consume it without sharing any part of the
computation they are compared on.

The paper's own structures (the aPF polymer and the NCCS carbon solid, and the TB parameter
sets of ASED / Cerda) are not available; the generators below stand in for them with carbon
systems of the same kind (sp3 diamond, sp2 graphite + sp3 grains, a dense disordered carbon),
each fully determined by its seed.

Units: Angstrom and eV.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GEOMETRY_SEED = 1210
SK_SEED = 1531
FD_SEED = 4

DIAMOND_A = 3.567          # conventional cubic lattice constant of diamond (Angstrom)
GRAPHITE_CC = 1.42         # in-plane C-C distance of graphite (Angstrom)
GRAPHITE_C2 = 3.35         # interlayer spacing of graphite (Angstrom)

# Fractional coordinates of the 8 atoms of the conventional diamond cell.
_DIAMOND_BASIS = np.array([
    [0.00, 0.00, 0.00], [0.00, 0.50, 0.50], [0.50, 0.00, 0.50], [0.50, 0.50, 0.00],
    [0.25, 0.25, 0.25], [0.25, 0.75, 0.75], [0.75, 0.25, 0.75], [0.75, 0.75, 0.25],
])


@dataclasses.dataclass(frozen=True)
class SKParams:
    """Numbers of a two-centre s/p Slater-Koster model (radial law chosen by the method code).

    Integral order everywhere: (ss-sigma, sp-sigma, pp-sigma, pp-pi).
    ``V0``/``S0`` are the values at ``r0``; ``qH``/``qS`` the exponential decay constants (1/A);
    ``r_on``..``r_cut`` is the interval of the smooth cutoff.
    """
    Es: float
    Ep: float
    V0: tuple
    qH: tuple
    S0: tuple
    qS: tuple
    r0: float = 1.54
    r_on: float = 2.3
    r_cut: float = 2.6

    def as_array(self) -> np.ndarray:
        """Packed float64[22]: Es, Ep, V0[4], qH[4], S0[4], qS[4], r0, r_on, r_cut, 0."""
        return np.array([self.Es, self.Ep, *self.V0, *self.qH, *self.S0, *self.qS,
                         self.r0, self.r_on, self.r_cut, 0.0], dtype=np.float64)


def sk_params(seed: int = SK_SEED) -> SKParams:
    """Seeded carbon-like parameter draw.

    Signs follow carbon: Vss_sigma < 0, Vsp_sigma > 0, Vpp_sigma > 0, Vpp_pi < 0, with every
    |V0| <= 6 eV. Each overlap integral has the sign opposite to its hopping, |S0| <= 0.25 at r0,
    and decays faster than the hopping (qS > qH). On-site energies Es = -5, Ep = +1 eV.
    """
    rng = np.random.default_rng(seed)
    sign = np.array([-1.0, 1.0, 1.0, -1.0])
    mag_v = np.array([rng.uniform(4.0, 6.0), rng.uniform(4.0, 6.0),
                      rng.uniform(4.0, 6.0), rng.uniform(1.0, 2.5)])
    V0 = sign * mag_v
    qH = rng.uniform(1.8, 2.4, size=4)
    mag_s = np.array([rng.uniform(0.08, 0.14), rng.uniform(0.08, 0.14),
                      rng.uniform(0.08, 0.14), rng.uniform(0.04, 0.08)])
    S0 = -sign * mag_s
    qS = qH + rng.uniform(0.2, 0.6, size=4)
    return SKParams(Es=-5.0, Ep=1.0, V0=tuple(V0.tolist()), qH=tuple(qH.tolist()),
                    S0=tuple(S0.tolist()), qS=tuple(qS.tolist()))


def _wrap(pos: np.ndarray, box: np.ndarray) -> np.ndarray:
    return pos - box * np.floor(pos / box)


def diamond(ncell, a: float = DIAMOND_A, sigma: float = 0.0, seed: int = GEOMETRY_SEED):
    """Diamond lattice of nx*ny*nz conventional cells with Gaussian displacements.

    Returns (pos float64[N,3] wrapped into [0, box), box float64[3]).
    Atom order: cells in C order (x slowest), 8 basis atoms per cell.
    """
    nx, ny, nz = ncell
    cells = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"),
                     axis=-1).reshape(-1, 3).astype(np.float64)
    pos = (cells[:, None, :] + _DIAMOND_BASIS[None, :, :]).reshape(-1, 3) * a
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    if sigma > 0.0:
        rng = np.random.default_rng(seed)
        pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    return _wrap(pos, box), box


def dimer(r: float, box_len: float = 40.0):
    """Two atoms separated by r along z in a large box (isolated molecule)."""
    box = np.full(3, box_len)
    c = box_len / 2
    pos = np.array([[c, c, c - r / 2], [c, c, c + r / 2]])
    return pos, box


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _graphite(ncell):
    """AB-stacked graphite in an orthorhombic cell a x a*sqrt(3) x 2c (8 atoms per cell)."""
    a = GRAPHITE_CC * math.sqrt(3.0)
    b = a * math.sqrt(3.0)
    c = 2.0 * GRAPHITE_C2
    layer_a = np.array([[0.0, 0.0], [a / 2, b / 6], [a / 2, b / 2], [0.0, 2 * b / 3]])
    layer_b = layer_a + np.array([0.0, GRAPHITE_CC])
    basis = np.concatenate([
        np.column_stack([layer_a, np.zeros(4)]),
        np.column_stack([layer_b, np.full(4, GRAPHITE_C2)]),
    ])
    nx, ny, nz = ncell
    cells = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"),
                     axis=-1).reshape(-1, 3).astype(np.float64)
    lat = np.array([a, b, c])
    pos = (cells[:, None, :] * lat + basis[None, :, :]).reshape(-1, 3)
    box = lat * np.array(ncell, dtype=np.float64)
    return _wrap(pos, box), box


def _min_image(d, box):
    return d - box * np.rint(d / box)


def _grain_sites(center, radius, rot, box):
    """Diamond lattice sites (a = 3.567) within `radius` of `center`, rotated by `rot`."""
    n = int(math.ceil(radius / DIAMOND_A)) + 1
    rng_c = np.arange(-n, n + 1, dtype=np.float64)
    cells = np.stack(np.meshgrid(rng_c, rng_c, rng_c, indexing="ij"), axis=-1).reshape(-1, 3)
    local = (cells[:, None, :] + _DIAMOND_BASIS[None, :, :]).reshape(-1, 3) * DIAMOND_A
    local = local[np.einsum("ij,ij->i", local, local) <= radius * radius]
    return _wrap(local @ rot.T + center, box)


def composite(n_atoms: int = 32768, seed: int = GEOMETRY_SEED, gap: float = 1.1,
              sigma: float = 0.05):
    """sp2-sp3 nano-composite carbon: seeded diamond grains (radius 8-15 A) in AB graphite.

    Graphite atoms within R + gap of a grain centre are replaced by the grain. The box is the
    smallest near-cubic graphite supercell (candidates in order of volume) for which the composite holds between
    n_atoms and 1.02*n_atoms atoms; the excess is then removed by deleting seeded-random graphite
    atoms (vacancies). Every atom is then displaced by seeded Gaussian noise of width `sigma`
    (a finite-temperature snapshot; perfect lattices leave whole symmetry sectors of a cluster
    decoupled, and the Krylov space of a column then picks up directions seeded by rounding).
    Returns (pos, box, is_grain bool[N]).
    """
    a = GRAPHITE_CC * math.sqrt(3.0)
    lat = np.array([a, a * math.sqrt(3.0), 2.0 * GRAPHITE_C2])
    side = (n_atoms / 0.13) ** (1.0 / 3.0)
    rng_n = [range(max(1, int(0.75 * side / l)), int(1.3 * side / l) + 2) for l in lat]
    cands = []
    for nx in rng_n[0]:
        for ny in rng_n[1]:
            for nz in rng_n[2]:
                dims = lat * np.array([nx, ny, nz])
                if dims.max() / dims.min() <= 1.3:
                    cands.append((float(np.prod(dims)), (nx, ny, nz)))
    cands.sort()
    for _, ncell in cands:
        g_pos, box = _graphite(ncell)
        if 8.0 * len(g_pos) < 0.9 * n_atoms * 8.0 * 0.8:
            continue
        rng = np.random.default_rng(seed)
        grains = []
        vol_target = 0.35 * float(np.prod(box))
        vol = 0.0
        tries = 0
        while vol < vol_target and tries < 2000:
            tries += 1
            radius = rng.uniform(8.0, 15.0)
            center = rng.uniform(0.0, 1.0, size=3) * box
            ok = 2 * radius + 2.0 <= box.min()
            for (c2, r2, _) in grains:
                if not ok:
                    break
                d = _min_image(center - c2, box)
                ok = np.linalg.norm(d) >= radius + r2 + 2.0
            if not ok:
                continue
            grains.append((center, radius, _random_rotation(rng)))
            vol += 4.0 / 3.0 * math.pi * radius ** 3
        keep = np.ones(len(g_pos), dtype=bool)
        parts = []
        for (center, radius, rot) in grains:
            d = _min_image(g_pos - center, box)
            keep &= np.einsum("ij,ij->i", d, d) > (radius + gap) ** 2
            parts.append(_grain_sites(center, radius, rot, box))
        grain_pos = np.concatenate(parts) if parts else np.zeros((0, 3))
        n_total = int(keep.sum()) + len(grain_pos)
        if n_atoms <= n_total <= int(1.02 * n_atoms):
            graphite_left = g_pos[keep]
            n_remove = n_total - n_atoms
            drop = rng.choice(len(graphite_left), size=n_remove, replace=False)
            mask = np.ones(len(graphite_left), dtype=bool)
            mask[drop] = False
            pos = np.concatenate([graphite_left[mask], grain_pos])
            is_grain = np.concatenate([np.zeros(int(mask.sum()), bool),
                                       np.ones(len(grain_pos), bool)])
            if sigma > 0.0:
                pos = _wrap(pos + np.random.default_rng(seed + 1).normal(0.0, sigma, pos.shape), box)
            return pos, box, is_grain
    raise RuntimeError("composite: no box size in the search range hit the atom count")


def amorphous(ncell=(64, 64, 32), density_gcc: float = 3.0, sigma: float = 0.3,
              dmin: float = 1.1, seed: int = GEOMETRY_SEED):
    """Dense disordered carbon: a diamond lattice scaled to `density_gcc`, displaced by
    Gaussian noise sigma; both atoms of every pair closer than `dmin` are redrawn (seeded)."""
    from scipy.spatial import cKDTree

    a = DIAMOND_A * (3.515 / density_gcc) ** (1.0 / 3.0)
    pos0, box = diamond(ncell, a=a, sigma=0.0)
    rng = np.random.default_rng(seed)
    disp = rng.normal(0.0, sigma, size=pos0.shape)
    for _ in range(100):
        pos = _wrap(pos0 + disp, box)
        tree = cKDTree(pos, boxsize=box)
        pairs = tree.query_pairs(dmin, output_type="ndarray")
        if len(pairs) == 0:
            return pos, box
        bad = np.unique(pairs.ravel())
        disp[bad] = rng.normal(0.0, sigma, size=(len(bad), 3))
    raise RuntimeError("amorphous: could not remove close pairs")


@dataclasses.dataclass
class Workload:
    """One synthetic system and the method settings it is run with."""
    name: str
    pos: np.ndarray
    box: np.ndarray
    sk: SKParams
    r_cluster: float        # <= 0: the cluster of every column is the whole system
    nu: int
    kT: float = 0.1
    electrons_per_atom: float = 4.0
    nu_classes: tuple = ()  # ((max_cluster_atoms, nu), ...) for size-dependent nu

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_electrons(self) -> float:
        return self.electrons_per_atom * self.n_atoms


def make(name: str) -> Workload:
    """The named synthetic workloads.

    diamond_64       64-atom diamond (2x2x2 cells), sigma 0.05 A, cluster = whole system, nu 30
    diamond_512      512-atom diamond (4x4x4 cells), sigma 0.1 A, cluster radius 6 A, nu 30: the
                     per-column work of diamond_4096 at an eighth of the columns (profiling size)
    diamond_4096     4096-atom diamond (8x8x8 cells), sigma 0.1 A, cluster radius 6 A, nu 30
    composite_32768  32768-atom graphite + diamond grains, cluster radius 6 A, nu 20/30/40 by size
                     (<= 100 cluster atoms: graphite interior; <= 140: grain boundaries; larger:
                     diamond grain interior)
    amorphous_1m     1,048,576-atom dense disordered carbon (3.0 g/cm3), cluster radius 5 A, nu 30
    """
    sk = sk_params()
    if name == "diamond_64":
        pos, box = diamond((2, 2, 2), sigma=0.05)
        return Workload(name, pos, box, sk, r_cluster=0.0, nu=30)
    if name == "diamond_512":
        pos, box = diamond((4, 4, 4), sigma=0.1)
        return Workload(name, pos, box, sk, r_cluster=6.0, nu=30)
    if name == "diamond_4096":
        pos, box = diamond((8, 8, 8), sigma=0.1)
        return Workload(name, pos, box, sk, r_cluster=6.0, nu=30)
    if name == "composite_32768":
        pos, box, _ = composite(32768)
        return Workload(name, pos, box, sk, r_cluster=6.0, nu=30,
                        nu_classes=((100, 20), (140, 30), (1 << 30, 40)))
    if name == "amorphous_1m":
        pos, box = amorphous()
        return Workload(name, pos, box, sk, r_cluster=5.0, nu=30)
    raise KeyError(name)


def fd_atoms(n_atoms: int, count: int = 32, seed: int = FD_SEED) -> np.ndarray:
    """Seeded choice of atoms for the finite-difference force check."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n_atoms, size=count, replace=False))


def sample_columns(n_columns: int, count: int, seed: int = GEOMETRY_SEED) -> np.ndarray:
    """Seeded sample of basis indices for checks at sizes the oracle cannot cover in full."""
    rng = np.random.default_rng(seed + 7)
    count = min(count, n_columns)
    return np.sort(rng.choice(n_columns, size=count, replace=False))
