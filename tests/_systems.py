"""Small seeded test systems shared by the oracle pins and the GPU parity tests."""
from __future__ import annotations

import os

import numpy as np

import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# Flat field offsets of one 14-field table record (m, gamma, lambda3, c, d, h, n,
# beta, lambda2, B, R, D, lambda1, A).
F_M, F_LAM3 = 0, 2


def table_for(names, mixer):
    elem, chi = W.element_records(names)
    return mixer(elem, chi)


def with_lambda3(table, lam3, m):
    t = np.array(table, dtype=np.float64).reshape(-1, 14).copy()
    t[:, F_LAM3] = lam3
    t[:, F_M] = m
    return t.ravel()


def si_cell(n=2, amp=0.12, seed=11):
    x, t, box = W.diamond(n, n, n, 5.432)
    rng = np.random.Generator(np.random.Philox(seed))
    return W.jitter_uniform(x, amp, rng), t, box


def sic_cell(n=2, sigma=0.12, seed=12, a=4.36):
    x, t, box = W.diamond(n, n, n, a, zincblende=True)
    rng = np.random.Generator(np.random.Philox(seed))
    return W.jitter_gaussian(x, sigma, rng), t, box


def packing_cell(n=64, c_frac=0.5, seed=13):
    rng = np.random.Generator(np.random.Philox(seed))
    x, t, box, ok = W.random_packing(n, c_frac, 2.3, 1.8, rng)
    assert ok
    return x, t, box


def read_cohesive():
    rows = []
    with open(os.path.join(GOLDEN, "cohesive_energies.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            s, sp, a, e, tol = line.split()
            rows.append((s, sp, float(a), float(e), float(tol)))
    return rows
