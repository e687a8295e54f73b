"""GB300 (sm_103a) Tersoff potential: energy, forces, virial and MD.

The compute path is the CUDA library ``libtersoff_gb300.so`` (C ABI in
``include/tersoff.h``); this package binds it (``Context``), builds the
per-triplet parameter table from element parameters (``params``), and wraps
energy and forces in a ``torch.autograd.Function`` whose backward is the
library's adjoint kernel (``autograd``).
"""
from ._lib import (  # noqa: F401
    Context,
    TersoffError,
    FP64,
    MIXED,
    SCATTER_GATHER,
    SCATTER_ATOMIC,
    NPARAM,
    NOALLOC_MAX_ATOMS,
    REBUILD_ON_SKIN,
    ABLATE_NO_SHORT,
    ABLATE_GENERAL,
    ABLATE_FP32_SUMS,
    ABLATE_FASTFWD,
    ABLATE_COMP_ATOM_SUMS,
    load,
    library_path,
    declared_symbols,
    pipe_peaks,
    checkpoint_info,
)
from .params import mix_tersoff89, read_table, write_table, FIELDS  # noqa: F401
from . import thermo  # noqa: F401
from .autograd import TersoffSystem, TersoffBatch, TersoffFunction, energy_forces  # noqa: F401
