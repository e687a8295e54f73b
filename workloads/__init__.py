"""Seeded synthetic inputs for the Tersoff benchmarks and tests.

This module produces input data only: lattices, displacements, velocities,
random packings, element parameter records and masses. It holds none of the
potential's arithmetic and is shared by the oracle tests, the GPU tests and the
benchmark, so both sides of every comparison see identical inputs.

The paper measures on "a standard LAMMPS benchmark" of crystalline silicon with
exactly four nearest neighbours per atom (Sec. VI). That input file is not
available; the diamond lattices below take its shape and stand in for it.
"""
from .synth import (  # noqa: F401
    rng_for,
    ELEMENTS_TERSOFF89,
    CHI_SIC,
    MASS_AMU,
    SEED_BASE,
    diamond,
    jitter_uniform,
    jitter_gaussian,
    maxwell_velocities,
    random_packing,
    batched_cells,
    batched_cell_sizes,
    element_records,
    config_si_small,
    config_si_md,
    config_sic,
    config_si_large,
)
