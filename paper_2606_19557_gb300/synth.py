"""Seeded synthetic structure batches shaped like the paper's training sets.

This module only builds geometry (lattices, strains, displacements, species
labels) and random parameter vectors.  It holds none of the NEP arithmetic and
is shared by the CUDA path's tests and benchmark and by the FP64 oracle's
tests, which both consume the arrays it returns.

The paper's datasets (carbon, water, PdCuNiP, the 16-element set, ...) are not
available, so seeded stand-ins are generated with the properties the paper
prints: structures of tens to hundreds of atoms (about 65 atoms on average in
the 16-element set, Sec. "Parameter optimization ... 16 elemental systems"),
solids, liquids and interfaces (Sec. "Training efficiency ... diverse
datasets").

Recipe (per structure):
  1. pick a lattice: FCC a = 3.6 A or BCC a = 2.87 A;
  2. build the smallest supercell with at least N sites, delete random sites
     down to N;
  3. apply a random symmetric strain with entries U(-strain, strain), which
     makes the cell triclinic;
  4. add Gaussian displacements of width sigma; resample displacements of
     atoms that come closer than 1.2 A to another atom or image;
  5. slabs: lengthen the third lattice vector by 10 A of vacuum;
  6. species uniform over the T types.
Positions are wrapped into the cell.  Rows of each 3x3 cell are the lattice
vectors (Angstrom).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

FCC_A = 3.6
BCC_A = 2.87
MIN_DIST = 1.2

_FCC_BASIS = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
_BCC_BASIS = np.array([[0, 0, 0], [0.5, 0.5, 0.5]])


@dataclasses.dataclass
class Batch:
    """A batch of periodic structures in CSR form.

    atom_off: int64 [Ns+1]; atoms of structure s are atom_off[s]:atom_off[s+1].
    pos:      float32 [Na, 3] Cartesian positions (Angstrom).
    types:    int32 [Na] species index in [0, n_types).
    cell:     float32 [Ns, 9] row-major 3x3 cells, rows = lattice vectors.
    """

    atom_off: np.ndarray
    pos: np.ndarray
    types: np.ndarray
    cell: np.ndarray
    n_types: int

    @property
    def n_struct(self) -> int:
        return int(self.atom_off.shape[0] - 1)

    @property
    def n_atoms(self) -> int:
        return int(self.atom_off[-1])

    def counts(self) -> np.ndarray:
        return np.diff(self.atom_off)

    def subset(self, idx) -> "Batch":
        """Structures idx (in that order) as a new batch."""
        idx = np.asarray(idx, dtype=np.int64)
        cnt = self.counts()[idx]
        off = np.zeros(len(idx) + 1, np.int64)
        off[1:] = np.cumsum(cnt)
        sel = np.concatenate([np.arange(self.atom_off[s], self.atom_off[s + 1]) for s in idx]) \
            if len(idx) else np.zeros(0, np.int64)
        return Batch(off, np.ascontiguousarray(self.pos[sel]), np.ascontiguousarray(self.types[sel]),
                     np.ascontiguousarray(self.cell[idx]), self.n_types)


def concat(batches) -> Batch:
    offs = [np.zeros(1, np.int64)]
    base = 0
    for b in batches:
        offs.append(b.atom_off[1:] + base)
        base += b.n_atoms
    return Batch(np.concatenate(offs), np.concatenate([b.pos for b in batches]),
                 np.concatenate([b.types for b in batches]),
                 np.concatenate([b.cell for b in batches]), max(b.n_types for b in batches))


def _supercell_reps(n_sites_per_cell: int, n: int):
    """Smallest n1*n2*n3 supercell with >= n sites, most cubic among ties."""
    best = None
    for n1 in range(1, 12):
        for n2 in range(n1, 12):
            for n3 in range(n2, 12):
                s = n1 * n2 * n3 * n_sites_per_cell
                if s < n:
                    continue
                key = (s, n3 - n1)
                if best is None or key < best[0]:
                    best = (key, (n1, n2, n3))
    if best is None:
        m = math.ceil((n / n_sites_per_cell) ** (1.0 / 3.0))
        return (m, m, m)
    return best[1]


def _lattice(kind: str, reps, a: float):
    basis = _FCC_BASIS if kind == "fcc" else _BCC_BASIS
    n1, n2, n3 = reps
    g = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1).reshape(-1, 3)
    frac = (g[:, None, :] + basis[None, :, :]).reshape(-1, 3) / np.array([n1, n2, n3], float)
    cell = np.diag([n1 * a, n2 * a, n3 * a]).astype(float)
    return frac, cell


def _close_atoms(pos: np.ndarray, cell: np.ndarray, dmin: float) -> np.ndarray:
    """Indices of atoms closer than dmin to another atom (minimum-image distances).

    The cells made here are orthorhombic up to a few per cent of strain and at least
    2 dmin wide, so rounding fractional differences finds the nearest image."""
    n = pos.shape[0]
    frac = pos @ np.linalg.inv(cell)
    if n > 300:
        return _close_atoms_tree(frac, cell, dmin)
    bad = np.zeros(n, bool)
    chunk = max(1, 4_000_000 // max(1, n))
    for i0 in range(0, n, chunk):
        i1 = min(n, i0 + chunk)
        df = frac[None, :, :] - frac[i0:i1, None, :]
        df -= np.round(df)
        d = df @ cell
        d2 = np.einsum("ijk,ijk->ij", d, d)
        idx = np.arange(i0, i1)
        d2[idx - i0, idx] = np.inf
        bad[i0:i1] |= (d2 < dmin * dmin).any(axis=1)
    return np.nonzero(bad)[0]


def _close_atoms_tree(frac: np.ndarray, cell: np.ndarray, dmin: float) -> np.ndarray:
    """Same result as the all-pairs check, for large cells: candidate pairs from a periodic
    k-d tree on the unstrained box (radius 1.2 dmin covers the few per cent of strain),
    then the exact minimum-image distance of each candidate."""
    from scipy.spatial import cKDTree
    f = frac - np.floor(frac)
    L = np.linalg.norm(cell, axis=1)
    x = np.minimum(f * L, np.nextafter(L, 0))
    pairs = cKDTree(x, boxsize=L).query_pairs(r=1.2 * dmin, output_type="ndarray")
    if pairs.size == 0:
        return np.zeros(0, np.int64)
    df = f[pairs[:, 1]] - f[pairs[:, 0]]
    df -= np.round(df)
    d = df @ cell
    close = pairs[np.einsum("ij,ij->i", d, d) < dmin * dmin]
    return np.unique(close.ravel())


def make_structure(rng: np.random.Generator, n: int, kind: str, strain: float, sigma: float,
                   n_types: int, slab: bool = False):
    """One structure: (pos [n,3], types [n], cell [3,3])."""
    if kind == "dimer":
        cell = np.eye(3) * 12.0
        r = rng.uniform(1.8, 3.2)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        c = np.full(3, 6.0)
        pos = np.stack([c - 0.5 * r * u, c + 0.5 * r * u])
        types = rng.integers(0, n_types, size=2)
        return pos, types.astype(np.int32), cell
    a = FCC_A if kind == "fcc" else BCC_A
    reps = _supercell_reps(4 if kind == "fcc" else 2, n)
    frac, cell = _lattice(kind, reps, a)
    if frac.shape[0] > n:
        keep = np.sort(rng.choice(frac.shape[0], size=n, replace=False))
        frac = frac[keep]
    if strain > 0:
        e = rng.uniform(-strain, strain, size=(3, 3))
        e = 0.5 * (e + e.T)
        cell = cell @ (np.eye(3) + e)
    pos0 = frac @ cell
    pos = pos0 + rng.normal(scale=sigma, size=pos0.shape)
    for _ in range(200):
        bad = _close_atoms(pos, cell, MIN_DIST)
        if bad.size == 0:
            break
        pos[bad] = pos0[bad] + rng.normal(scale=sigma, size=(bad.size, 3))
    else:
        raise RuntimeError("could not place atoms at least 1.2 A apart")
    if slab:
        c = cell[2]
        cell = cell.copy()
        cell[2] = c * (1.0 + 10.0 / np.linalg.norm(c))
    # wrap positions into the (possibly enlarged) cell
    f = pos @ np.linalg.inv(cell)
    f -= np.floor(f)
    pos = f @ cell
    types = rng.integers(0, n_types, size=pos.shape[0])
    return pos, types.astype(np.int32), cell


def _assemble(structs, n_types: int) -> Batch:
    counts = np.array([p.shape[0] for p, _, _ in structs], np.int64)
    off = np.zeros(len(structs) + 1, np.int64)
    off[1:] = np.cumsum(counts)
    pos = np.concatenate([p for p, _, _ in structs]).astype(np.float32) if structs else np.zeros((0, 3), np.float32)
    types = np.concatenate([t for _, t, _ in structs]).astype(np.int32) if structs else np.zeros(0, np.int32)
    cell = np.stack([c.reshape(9) for _, _, c in structs]).astype(np.float32) if structs else np.zeros((0, 9), np.float32)
    return Batch(off, np.ascontiguousarray(pos), types, np.ascontiguousarray(cell), n_types)


# --------------------------------------------------------------------------------------------
# Model configurations (NEP input-file keys of Table 1: type, cutoff, n_max, basis_size, l_max,
# neuron).  has_4b / has_5b stand for the second and third entries of l_max ("4 2 1").
# --------------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class ModelSpec:
    n_types: int
    rc_R: float
    rc_A: float
    n_max_R: int
    n_max_A: int
    basis_R: int
    basis_A: int
    l_max: int
    has_4b: int
    has_5b: int
    n_neu: int


SPECS = {
    "fcc32_t1": ModelSpec(1, 5.0, 4.0, 4, 4, 8, 8, 4, 0, 0, 10),
    "fcc_bcc_t1": ModelSpec(1, 6.0, 4.0, 4, 4, 8, 8, 4, 1, 0, 30),
    "alloy_t4": ModelSpec(4, 6.0, 4.0, 4, 4, 8, 8, 4, 1, 0, 30),
    "scale_t5": ModelSpec(5, 6.0, 4.0, 6, 6, 10, 10, 4, 1, 1, 50),
    # Table 1 carbon input: cutoff 4.2 3.7, n_max 10 8, basis 10 8, l_max 4 2 1, 100 neurons
    "carbon_table1": ModelSpec(1, 4.2, 3.7, 10, 8, 10, 8, 4, 1, 1, 100),
    # Table 2 16-element models NEP44 / NEP88 (70,401 / 124,673 parameters); the cutoffs are
    # not printed with them, 6 / 4 A as in the other configurations
    "nep44_t16": ModelSpec(16, 6.0, 4.0, 4, 4, 8, 8, 4, 1, 1, 80),
    "nep88_t16": ModelSpec(16, 6.0, 4.0, 8, 8, 8, 8, 4, 1, 1, 80),
}


def batch_fcc32(seed: int = 1, n_struct: int = 8) -> Batch:
    """8 FCC 2x2x2 cells (32 atoms, a = 3.6 A), Gaussian displacements 0.1 A, 1 species."""
    rng = np.random.default_rng(seed)
    structs = [make_structure(rng, 32, "fcc", 0.0, 0.1, 1) for _ in range(n_struct)]
    return _assemble(structs, 1)


def batch_fcc_bcc(seed: int = 2, n_struct: int = 1000, n_lo: int = 64, n_hi: int = 256,
                  n_types: int = 1) -> Batch:
    """FCC/BCC supercells of U{n_lo..n_hi} atoms, strain +-3 %, sigma U(0.05, 0.3) A."""
    rng = np.random.default_rng(seed)
    structs = []
    for _ in range(n_struct):
        n = int(rng.integers(n_lo, n_hi + 1))
        kind = "fcc" if rng.random() < 0.5 else "bcc"
        sigma = rng.uniform(0.05, 0.3)
        structs.append(make_structure(rng, n, kind, 0.03, sigma, n_types))
    return _assemble(structs, n_types)


def batch_alloy(seed: int = 3, n_struct: int = 5000, n_types: int = 4, n_lo: int = 16,
                n_hi: int = 512) -> Batch:
    """Random alloy: 20 % liquid-like (sigma 0.5 A), 10 % slabs (+10 A vacuum), rest as above."""
    rng = np.random.default_rng(seed)
    structs = []
    for _ in range(n_struct):
        n = int(rng.integers(n_lo, n_hi + 1))
        kind = "fcc" if rng.random() < 0.5 else "bcc"
        u = rng.random()
        if u < 0.2:
            structs.append(make_structure(rng, n, kind, 0.03, 0.5, n_types))
        elif u < 0.3:
            structs.append(make_structure(rng, n, kind, 0.03, rng.uniform(0.05, 0.3), n_types, slab=True))
        else:
            structs.append(make_structure(rng, n, kind, 0.03, rng.uniform(0.05, 0.3), n_types))
    return _assemble(structs, n_types)


def _scale_structure(seed: int, s: int, n_struct: int, n_types: int, big_atoms: int):
    """Structure s of the scale batch, from its own random stream (seed, s): structures
    s < n_struct have log-uniform sizes in [2, 2000], the rest are large FCC cells."""
    rng = np.random.default_rng([seed, s])
    if s >= n_struct:
        return make_structure(rng, big_atoms, "fcc", 0.03, rng.uniform(0.05, 0.3), n_types)
    n = int(round(math.exp(rng.uniform(math.log(2), math.log(2000)))))
    if n <= 2:
        return make_structure(rng, 2, "dimer", 0.0, 0.0, n_types)
    kind = "fcc" if rng.random() < 0.5 else "bcc"
    u = rng.random()
    sigma = 0.5 if u < 0.2 else rng.uniform(0.05, 0.3)
    return make_structure(rng, n, kind, 0.03, sigma, n_types, slab=(0.2 <= u < 0.3))


def _scale_chunk(args):
    seed, idx, n_struct, n_types, big_atoms = args
    return [_scale_structure(seed, int(s), n_struct, n_types, big_atoms) for s in idx]


def batch_scale(seed: int = 5, n_struct: int = 20000, n_types: int = 5, n_big: int = 10,
                big_atoms: int = 10000, only=None, workers: int = 0) -> Batch:
    """Sizes log-uniform in [2, 2000] (2 atoms: a dimer in a 12 A cubic cell) plus n_big
    large FCC cells (indices n_struct .. n_struct + n_big - 1).

    Every structure draws from its own stream (seed, index), so `only` (a list of
    indices) builds exactly those structures of the full batch, in that order, without
    the others.  workers > 1 spreads the structures over that many spawned processes."""
    idx = np.arange(n_struct + n_big) if only is None else np.asarray(only, np.int64)
    if workers > 1 and idx.size > 256:
        import concurrent.futures
        import multiprocessing
        parts = np.array_split(idx, 4 * workers)
        ctx = multiprocessing.get_context("spawn")
        with concurrent.futures.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
            chunks = ex.map(_scale_chunk, [(seed, p, n_struct, n_types, big_atoms) for p in parts])
            structs = [st for ch in chunks for st in ch]
    else:
        structs = _scale_chunk((seed, idx, n_struct, n_types, big_atoms))
    return _assemble(structs, n_types)


def random_theta(n_params: int, seed: int, lo: float = -0.5, hi: float = 0.5) -> np.ndarray:
    """Parameter vector drawn U(lo, hi) (float32 values, returned as float64)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n_params).astype(np.float32).astype(np.float64)


def random_targets(batch: Batch, seed: int, e_per_atom: float = 1.0, f_scale: float = 1.0,
                   w_per_atom: float = 1.0):
    """Seeded reference values (E [Ns] f64, F [Na,3] f32, W [Ns,9] f64) with the shapes of DFT labels."""
    rng = np.random.default_rng(seed)
    cnt = batch.counts().astype(np.float64)
    E = rng.normal(scale=e_per_atom, size=batch.n_struct) * cnt
    F = rng.normal(scale=f_scale, size=(batch.n_atoms, 3)).astype(np.float32)
    W = rng.normal(scale=w_per_atom, size=(batch.n_struct, 9)) * cnt[:, None]
    W = 0.5 * (W + W.reshape(-1, 3, 3).transpose(0, 2, 1).reshape(-1, 9))
    return E, F, W
