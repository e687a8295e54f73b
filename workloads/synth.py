"""Seeded synthetic structures (positions, species, boxes, velocities).

Everything here is input data. Random numbers come from numpy's Philox
generator seeded with ``SEED_BASE + k`` so every consumer draws the same
stream. Units are LAMMPS "metal": Angstrom, ps, amu, eV, K.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1607029040

# Tersoff, Phys. Rev. B 39, 5566 (1989), Table I: per-element records
# (A [eV], B [eV], lambda [1/A], mu [1/A], beta, n, c, d, h, R [A], S [A]).
# R and S are the inner and outer radii of the cutoff function.
ELEMENTS_TERSOFF89 = {
    "Si": (1830.8, 471.18, 2.4799, 1.7322, 1.1e-6, 0.78734, 1.0039e5, 16.217,
           -0.59825, 2.7, 3.0),
    "C": (1393.6, 346.74, 3.4879, 2.2119, 1.5724e-7, 0.72751, 3.8049e4, 4.3484,
          -0.57058, 1.8, 2.1),
}
# Tersoff (1989): chi for the Si-C pair.
CHI_SIC = 0.9776

MASS_AMU = {"Si": 28.0855, "C": 12.011}

# Unit constants used to draw Maxwell velocities (metal units).
_KB_EV = 8.617333262e-5          # Boltzmann constant, eV/K
_MVV2E = 1.0364269e-4            # 1 amu A^2/ps^2 in eV
_AMU_G = 1.66053906660           # 1 amu / (1 g/cm^3 * 1 A^3) ... 1 amu = 1.66054e-24 g

_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
_DIAMOND_BASIS = np.concatenate([_FCC, _FCC + 0.25])


def rng_for(k: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(SEED_BASE + int(k)))


def element_records(names):
    """(ns x 11) element records and the (ns x ns) chi matrix for ``names``."""
    elem = np.array([ELEMENTS_TERSOFF89[s] for s in names], dtype=np.float64)
    ns = len(names)
    chi = np.ones((ns, ns), dtype=np.float64)
    for a in range(ns):
        for b in range(ns):
            if {names[a], names[b]} == {"Si", "C"}:
                chi[a, b] = CHI_SIC
    return elem, chi


def diamond(nx: int, ny: int, nz: int, a: float, zincblende: bool = False):
    """Diamond (or zincblende) lattice of nx*ny*nz cubic cells, 8 atoms each.

    Atoms are ordered cell by cell (x fastest), basis order inside a cell.
    With ``zincblende`` the fcc sub-lattice is species 0 and the (1/4,1/4,1/4)
    sub-lattice species 1. Returns (x [N,3] float64, types [N] int32, box [3]).
    """
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    origins = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    x = (origins[:, None, :] + _DIAMOND_BASIS[None, :, :]).reshape(-1, 3) * a
    t = np.zeros((origins.shape[0], 8), dtype=np.int32)
    if zincblende:
        t[:, 4:] = 1
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    return np.ascontiguousarray(x), t.ravel(), box


def jitter_uniform(x: np.ndarray, amp: float, rng: np.random.Generator) -> np.ndarray:
    return x + rng.uniform(-amp, amp, size=x.shape)


def jitter_gaussian(x: np.ndarray, sigma: float, rng: np.random.Generator) -> np.ndarray:
    return x + rng.normal(0.0, sigma, size=x.shape)


def maxwell_velocities(types: np.ndarray, masses: np.ndarray, temp: float,
                       rng: np.random.Generator) -> np.ndarray:
    """Maxwell-Boltzmann velocities (A/ps) at ``temp`` K, zero net momentum."""
    m = np.asarray(masses, dtype=np.float64)[types]
    sig = np.sqrt(_KB_EV * temp / (m * _MVV2E))
    v = rng.normal(0.0, 1.0, size=(types.shape[0], 3)) * sig[:, None]
    p = (m[:, None] * v).sum(axis=0) / m.sum()
    return np.ascontiguousarray(v - p[None, :])


def random_packing(n: int, c_frac: float, density_gcc: float, min_sep: float,
                   rng: np.random.Generator, max_batches: int = 20000):
    """Random sequential insertion of ``n`` Si/C atoms in a periodic cube.

    Species: C with probability ``c_frac`` per atom (type 1), else Si (type 0).
    The cube's volume gives the mass density ``density_gcc``; every pair of
    atoms is at least ``min_sep`` apart (minimum image). Candidates are drawn
    in batches; a candidate is accepted, in draw order, when no atom placed
    before it (earlier batches: a periodic k-d tree query; its own batch: a
    direct check) is closer than ``min_sep``. Returns (x, types, box, ok);
    ``ok`` is False when the attempt budget ran out.
    """
    from scipy.spatial import cKDTree

    types = (rng.random(n) < c_frac).astype(np.int32)
    masses = np.where(types == 1, MASS_AMU["C"], MASS_AMU["Si"])
    vol = masses.sum() * _AMU_G / density_gcc  # A^3
    L = vol ** (1.0 / 3.0)
    pos = np.zeros((n, 3), dtype=np.float64)
    placed = 0
    s2 = min_sep * min_sep
    batch = 1024
    for _ in range(max_batches):
        if placed == n:
            break
        cand = rng.random((batch, 3)) * L
        if placed:
            tree = cKDTree(pos[:placed], boxsize=L)
            dist, _ = tree.query(cand, k=1, distance_upper_bound=min_sep)
            surv = np.nonzero(dist >= min_sep)[0]
        else:
            surv = np.arange(batch)
        if surv.size == 0:
            continue
        cs = cand[surv]
        d = cs[:, None, :] - cs[None, :, :]
        d -= L * np.rint(d / L)
        near = (d * d).sum(axis=2) < s2
        np.fill_diagonal(near, False)
        taken = np.zeros(surv.size, dtype=bool)
        for k in range(surv.size):
            if placed == n:
                break
            if near[k, taken].any():
                continue
            pos[placed] = cs[k]
            placed += 1
            taken[k] = True
    box = np.array([L, L, L], dtype=np.float64)
    return np.ascontiguousarray(pos[:placed]), types[:placed], box, placed == n


def _batched_cell(args):
    c, size, frac, density_gcc, min_sep, seed_k = args
    k = 0
    while True:
        r = np.random.Generator(np.random.Philox([SEED_BASE + seed_k, c, k]))
        x, t, box, ok = random_packing(int(size), float(frac), density_gcc, min_sep, r)
        if ok:
            return x, t, box
        k += 1


def batched_cell_sizes(n_cells: int = 256, nmin: int = 64, nmax: int = 4096, seed_k: int = 4):
    """Atom counts and C fractions of the batched workload's cells (the draws
    that precede the packings), without generating the packings."""
    rng = rng_for(seed_k)
    sizes = rng.integers(nmin, nmax + 1, size=n_cells)
    fracs = rng.random(n_cells)
    return sizes, fracs


def batched_cells(n_cells: int = 256, nmin: int = 64, nmax: int = 4096,
                  density_gcc: float = 2.3, min_sep: float = 1.8, seed_k: int = 4,
                  map_fn=map, subset=None):
    """Independent periodic Si/C cells of uneven size for the batched workload.

    Atom counts ~ U{nmin..nmax}, C fraction ~ U(0,1) per cell; each cell is a
    random packing at ``density_gcc`` with minimum separation ``min_sep``. A
    cell whose packing runs out of attempts is drawn again from the next seed.
    Every cell has its own generator, so ``map_fn`` may be a process pool's map
    and ``subset`` (cell indices) generates only those cells, identical to
    their counterparts in the whole batch.
    """
    sizes, fracs = batched_cell_sizes(n_cells, nmin, nmax, seed_k)
    cells = range(n_cells) if subset is None else subset
    jobs = [(c, sizes[c], fracs[c], density_gcc, min_sep, seed_k) for c in cells]
    return list(map_fn(_batched_cell, jobs))


# --------------------------------------------------------------------- named workloads
def config_si_small():
    """Si diamond 8x8x8 cells (4,096 atoms, a = 5.432 A), uniform jitter +-0.1 A."""
    x, t, box = diamond(8, 8, 8, 5.432)
    x = jitter_uniform(x, 0.1, rng_for(1))
    return x, t, box, ["Si"]


def config_si_md(ncell: int = 40, temp: float = 1000.0):
    """Si diamond ncell^3 cells, Gaussian sigma 0.05 A, Maxwell velocities."""
    x, t, box = diamond(ncell, ncell, ncell, 5.432)
    rng = rng_for(2)
    x = jitter_gaussian(x, 0.05, rng)
    v = maxwell_velocities(t, np.array([MASS_AMU["Si"]]), temp, rng)
    return x, v, t, box, ["Si"]


def config_sic(ncell: int = 64, a: float = 4.36):
    """SiC zincblende ncell^3 cells, Gaussian sigma 0.08 A."""
    x, t, box = diamond(ncell, ncell, ncell, a, zincblende=True)
    x = jitter_gaussian(x, 0.08, rng_for(3))
    return x, t, box, ["Si", "C"]


def config_si_large(nx: int = 160, ny: int = 160, nz: int = 80, temp: float = 1000.0):
    """Si diamond 160x160x80 cells (16,384,000 atoms), Maxwell velocities."""
    x, t, box = diamond(nx, ny, nz, 5.432)
    rng = rng_for(5)
    x = jitter_gaussian(x, 0.05, rng)
    v = maxwell_velocities(t, np.array([MASS_AMU["Si"]]), temp, rng)
    return x, v, t, box, ["Si"]
