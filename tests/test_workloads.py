"""The seeded input generators (workloads/synth.py) against the recipe they
state: lattice geometry, the packings' minimum separation and density, the
velocities' temperature and momentum, and the batched cells' sizes, boxes
and determinism. CPU only.
"""
import numpy as np

import oracle
import workloads as W


def test_diamond_lattice_geometry():
    x, t, box = W.diamond(3, 2, 4, 5.432)
    assert x.shape == (3 * 2 * 4 * 8, 3) and np.allclose(box, [3 * 5.432, 2 * 5.432, 4 * 5.432])
    cnt, nbr = oracle.neighbors(x, box, 2.5)
    assert np.all(cnt == 4)  # four nearest neighbours at a sqrt(3)/4
    d = x[nbr[:, :4]] - x[:, None, :]
    d -= box * np.round(d / box)
    assert np.allclose(np.sqrt((d * d).sum(-1)), 5.432 * np.sqrt(3) / 4, atol=1e-12)
    _, tz, _ = W.diamond(2, 2, 2, 4.36, zincblende=True)
    assert (tz == 1).sum() == (tz == 0).sum() == 32


def test_random_packing_separation_and_density():
    rng = W.rng_for(200)
    x, t, box, ok = W.random_packing(400, 0.5, 2.3, 1.8, rng)
    assert ok and len(x) == 400
    d = x[:, None, :] - x[None, :, :]
    d -= box * np.round(d / box)
    r = np.sqrt((d * d).sum(-1)) + np.eye(len(x)) * 1e9
    assert r.min() >= 1.8
    mass = np.where(t == 1, W.MASS_AMU["C"], W.MASS_AMU["Si"]).sum()
    rho = mass * 1.66053906660 / box.prod()  # g/cm^3
    assert abs(rho - 2.3) < 1e-9
    assert np.all(box == box[0]) and np.all((x >= 0) & (x < box))


def test_maxwell_velocities_temperature_and_momentum():
    x, t, box = W.diamond(10, 10, 10, 5.432)
    m = np.array([W.MASS_AMU["Si"]])
    v = W.maxwell_velocities(t, m, 1000.0, W.rng_for(201))
    p = (m[t][:, None] * v).sum(axis=0)
    assert np.abs(p).max() < 1e-9
    kb, mvv2e = 8.617333262e-5, 1.0364269e-4  # eV/K; eV per amu A^2/ps^2
    temp = (m[t][:, None] * v * v).sum() * mvv2e / (3 * len(t) * kb)
    assert abs(temp - 1000.0) < 30.0  # 8,000 atoms: ~1% statistical spread


def test_batched_cells_recipe():
    a = W.batched_cells(n_cells=12, nmin=64, nmax=600, seed_k=202)
    b = W.batched_cells(n_cells=12, nmin=64, nmax=600, seed_k=202)
    for (xa, ta, ba), (xb, tb, bb) in zip(a, b):
        assert np.array_equal(xa, xb) and np.array_equal(ta, tb) and np.array_equal(ba, bb)
    sizes = np.array([len(c[0]) for c in a])
    assert sizes.min() >= 64 and sizes.max() <= 600
    # every box admits the 4.0 A list radius (edges of at least 8 A)
    assert min(c[2].min() for c in a) >= 8.0
    # the smallest possible cell: 64 C atoms at 2.3 g/cm^3
    x, t, box, ok = W.random_packing(64, 1.0, 2.3, 1.8, W.rng_for(203))
    assert ok and box[0] >= 8.0
